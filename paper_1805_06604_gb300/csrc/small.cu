// small.cu -- the O((m+n) r^2) and O(mn)-once kernels of an outer iteration.
//
//  * ||X||_F^2 (Remark 1's constant term), FP64, once at creation.
//  * Grams G = W^T W and D = H H^T (the W(:,k)^T W(:,j) coefficients of the
//    HALS closed form, Sec. 1), split over the long dimension with one
//    partial per CTA and a fixed-order second pass (deterministic).
//  * e(0) of Algorithm 2 step 1 through Remark 1.
//  * The finalize kernel of Algorithm 2 steps 11-20: W_y = W_n + beta (W_n - W)
//    (optionally projected), H_y for hp = 1, and the accept / restart copies,
//    driven by the decision the W-sweep kernel left in the device state.
#include <cuda_runtime.h>
#include <math.h>

#include "common.cuh"

namespace nmfg {
namespace {

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <int NT>
__device__ double block_sum_d(double v, double *red) {
    v = warp_sum_d(v);
    const int w = threadIdx.x / 32, l = threadIdx.x % 32;
    if (l == 0) red[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < NT / 32; ++i) s += red[i];
    __syncthreads();
    return s;   // valid in thread 0
}

// Kahan's compensated addition: (sum, c) absorbs v; sum - c is the result.
__device__ __forceinline__ void kahan_add(float &sum, float &c, float v) {
    const float y = v - c;
    const float t = sum + y;
    c = (t - sum) - y;
    sum = t;
}

// Error-free transformations: a*b = p + e exactly (FMA), a+b = s + e exactly.
__device__ __forceinline__ void two_prod(float a, float b, float &p, float &e) {
    p = a * b;
    e = fmaf(a, b, -p);
}
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

constexpr int kRedThreads = 256;
constexpr int kRedBlocks = 2 * kNumSMs;

// ---------------------------------------------------------------- ||X||^2
__global__ void __launch_bounds__(kRedThreads)
fro2_partial_kernel(const float *__restrict__ v, int64_t rows, int64_t cols, int64_t ld,
                    double *__restrict__ part) {
    __shared__ double red[kRedThreads / 32];
    double acc = 0.0;
    const int64_t total = rows * cols;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = q / cols, j = q % cols;
        const double x = (double)v[i * ld + j];
        acc = fma(x, x, acc);
    }
    const double s = block_sum_d<kRedThreads>(acc, red);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void sum_partials_kernel(const double *__restrict__ part, int count,
                                    double *__restrict__ out) {
    __shared__ double red[kRedThreads / 32];
    double acc = 0.0;
    for (int i = threadIdx.x; i < count; i += blockDim.x) acc += part[i];
    const double s = block_sum_d<kRedThreads>(acc, red);
    if (threadIdx.x == 0) *out = s;
}

// ---------------------------------------------------------------- Grams
// Partial Gram of a chunk of the long dimension.  Thread (ty, tx) of a
// 16 x 16 block owns entries (ty + 16a, tx + 16b), a, b < RB (R = 16 RB).
// ROWS = true: M is N x ldm (entries M[i*ldm + k], k < r), G = M^T M.
// ROWS = false: M is r x ldm (entries M[k*ldm + i], i < N), G = M M^T.
constexpr int GBK = 32;

// EXACT = false: 32-row blocks summed in FP32, blocks combined with Kahan's
// correction (the Gram feeds the sweeps; FP32 accuracy).  EXACT = true: every
// product and sum goes through an error-free transformation and the result
// is kept as an unevaluated pair hi + lo (the Gram of H_y also feeds the
// Remark 1 error, whose cancellation needs it to about 2^-40 relative).
template <int RB, bool ROWS, bool EXACT>
__device__ __forceinline__ void
gram_partial_body(const float *__restrict__ M, int64_t N, int64_t ldm, int r, int64_t chunk,
                  float *__restrict__ part, float *__restrict__ part_lo, int rs, int64_t bid) {
    constexpr int R = 16 * RB;
    __shared__ float Ms[GBK][R + 1];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const int64_t i0 = bid * chunk;
    const int64_t i1 = min(N, i0 + chunk);
    float acc[RB][RB], comp[RB][RB];
#pragma unroll
    for (int a = 0; a < RB; ++a)
#pragma unroll
        for (int b = 0; b < RB; ++b) acc[a][b] = comp[a][b] = 0.0f;

    for (int64_t ib = i0; ib < i1; ib += GBK) {
        for (int idx = threadIdx.x; idx < GBK * R; idx += 256) {
            int ii, k;
            if (ROWS) {
                ii = idx / R;
                k = idx % R;
            } else {
                k = idx / GBK;
                ii = idx % GBK;
            }
            const int64_t i = ib + ii;
            float v = 0.0f;
            if (i < i1 && k < r) v = ROWS ? M[i * ldm + k] : M[(int64_t)k * ldm + i];
            Ms[ii][k] = v;
        }
        __syncthreads();
        if constexpr (EXACT) {
#pragma unroll 2
            for (int ii = 0; ii < GBK; ++ii) {
                float va[RB], vb[RB];
#pragma unroll
                for (int a = 0; a < RB; ++a) va[a] = Ms[ii][ty + 16 * a];
#pragma unroll
                for (int b = 0; b < RB; ++b) vb[b] = Ms[ii][tx + 16 * b];
#pragma unroll
                for (int a = 0; a < RB; ++a)
#pragma unroll
                    for (int b = 0; b < RB; ++b) {
                        float p, pe, s, se;
                        two_prod(va[a], vb[b], p, pe);
                        two_sum(acc[a][b], p, s, se);
                        acc[a][b] = s;
                        comp[a][b] += se + pe;       // comp = low-order part
                    }
            }
        } else {
            float blk[RB][RB];
#pragma unroll
            for (int a = 0; a < RB; ++a)
#pragma unroll
                for (int b = 0; b < RB; ++b) blk[a][b] = 0.0f;
#pragma unroll 4
            for (int ii = 0; ii < GBK; ++ii) {
                float va[RB], vb[RB];
#pragma unroll
                for (int a = 0; a < RB; ++a) va[a] = Ms[ii][ty + 16 * a];
#pragma unroll
                for (int b = 0; b < RB; ++b) vb[b] = Ms[ii][tx + 16 * b];
#pragma unroll
                for (int a = 0; a < RB; ++a)
#pragma unroll
                    for (int b = 0; b < RB; ++b) blk[a][b] = fmaf(va[a], vb[b], blk[a][b]);
            }
#pragma unroll
            for (int a = 0; a < RB; ++a)
#pragma unroll
                for (int b = 0; b < RB; ++b) kahan_add(acc[a][b], comp[a][b], blk[a][b]);
        }
        __syncthreads();
    }
    float *out = part + bid * rs * rs;
#pragma unroll
    for (int a = 0; a < RB; ++a)
#pragma unroll
        for (int b = 0; b < RB; ++b) {
            const int i = ty + 16 * a, j = tx + 16 * b;
            if (i < rs && j < rs) {
                if constexpr (EXACT) {
                    out[i * rs + j] = acc[a][b];
                    part_lo[bid * rs * rs + i * rs + j] = comp[a][b];
                } else {
                    out[i * rs + j] = acc[a][b] - comp[a][b];
                }
            }
        }
}

template <int RB, bool ROWS, bool EXACT>
__global__ void __launch_bounds__(256)
gram_partial_kernel(const float *__restrict__ M, int64_t N, int64_t ldm, int r,
                    int64_t chunk, float *__restrict__ part, float *__restrict__ part_lo, int rs) {
    gram_partial_body<RB, ROWS, EXACT>(M, N, ldm, r, chunk, part, part_lo, rs, blockIdx.x);
}
template <int RB, bool ROWS, bool EXACT>
__global__ void __launch_bounds__(256)
gram_partial_grouped(const GramItem *__restrict__ items, const int64_t *__restrict__ begin,
                     int nitems) {
    int64_t local;
    const GramItem &it = items[group_item(begin, nitems, local)];
    gram_partial_body<RB, ROWS, EXACT>(it.M, it.N, it.ldm, it.r, it.chunk, it.part, it.part_lo,
                                       it.rs, local);
}

// Sum of the per-chunk partial Grams.  A CTA owns 32 consecutive entries
// (one per lane, so each load is one coalesced row of a partial); its eight
// warps take the partials p = w, w + 8, ... (independent loads in flight),
// and the eight warp sums are combined in warp order (deterministic).
constexpr int kRedWarps = 8;

__device__ __forceinline__ void gram_reduce_body(const float *__restrict__ part, int nparts,
                                                 int rs, float *__restrict__ G, int bid) {
    __shared__ float sh[kRedWarps][32], sc[kRedWarps][32];
    const int lane = threadIdx.x % 32, w = threadIdx.x / 32;
    const int e = bid * 32 + lane;
    const int ne = rs * rs;
    float s = 0.0f, c = 0.0f;
    if (e < ne) {
#pragma unroll 4
        for (int p = w; p < nparts; p += kRedWarps) kahan_add(s, c, part[(int64_t)p * ne + e]);
    }
    sh[w][lane] = s;
    sc[w][lane] = c;
    __syncthreads();
    if (w == 0 && e < ne) {
        float t = 0.0f, tc = 0.0f;
        for (int q = 0; q < kRedWarps; ++q) {
            kahan_add(t, tc, sh[q][lane]);
            kahan_add(t, tc, -sc[q][lane]);
        }
        G[e] = t - tc;
    }
}

// Pairs (hi_p, lo_p) summed exactly into G + G_lo (hi part rounded to FP32),
// with the same decomposition.
__device__ __forceinline__ void gram_reduce_exact_body(const float *__restrict__ part,
                                                       const float *__restrict__ part_lo,
                                                       int nparts, int rs,
                                                       float *__restrict__ G,
                                                       float *__restrict__ G_lo, int bid) {
    __shared__ float sh[kRedWarps][32], sl[kRedWarps][32];
    const int lane = threadIdx.x % 32, w = threadIdx.x / 32;
    const int e = bid * 32 + lane;
    const int ne = rs * rs;
    float hi = 0.0f, lo = 0.0f;
    if (e < ne) {
#pragma unroll 4
        for (int p = w; p < nparts; p += kRedWarps) {
            float s, se;
            two_sum(hi, part[(int64_t)p * ne + e], s, se);
            hi = s;
            lo += se + part_lo[(int64_t)p * ne + e];
        }
    }
    sh[w][lane] = hi;
    sl[w][lane] = lo;
    __syncthreads();
    if (w == 0 && e < ne) {
        float th = 0.0f, tl = 0.0f;
        for (int q = 0; q < kRedWarps; ++q) {
            float s, se;
            two_sum(th, sh[q][lane], s, se);
            th = s;
            tl += se + sl[q][lane];
        }
        float g, ge;
        two_sum(th, tl, g, ge);
        G[e] = g;
        G_lo[e] = ge;
    }
}

__global__ void __launch_bounds__(kRedWarps * 32)
gram_reduce_kernel(const float *__restrict__ part, int nparts, int rs, float *__restrict__ G) {
    gram_reduce_body(part, nparts, rs, G, blockIdx.x);
}
__global__ void __launch_bounds__(kRedWarps * 32)
gram_reduce_exact_kernel(const float *__restrict__ part, const float *__restrict__ part_lo,
                         int nparts, int rs, float *__restrict__ G, float *__restrict__ G_lo) {
    gram_reduce_exact_body(part, part_lo, nparts, rs, G, G_lo, blockIdx.x);
}
template <bool EXACT>
__global__ void __launch_bounds__(kRedWarps * 32)
gram_reduce_grouped(const GramItem *__restrict__ items, const int64_t *__restrict__ begin,
                    int nitems) {
    int64_t local;
    const GramItem &it = items[group_item(begin, nitems, local)];
    if constexpr (EXACT)
        gram_reduce_exact_body(it.part, it.part_lo, it.nparts, it.rs, it.G, it.G_lo, (int)local);
    else
        gram_reduce_body(it.part, it.nparts, it.rs, it.G, (int)local);
}

struct GramPlan {
    int nparts;
    int64_t chunk;
};

// Chunks of whole 32-row blocks, about two CTAs per SM at most.
GramPlan plan_gram(int64_t N) {
    GramPlan p;
    int64_t want = (N + GBK - 1) / GBK;
    if (want > 2 * kNumSMs) want = 2 * kNumSMs;
    if (want < 1) want = 1;
    p.chunk = ((N + want - 1) / want + GBK - 1) / GBK * GBK;
    p.nparts = (int)((N + p.chunk - 1) / p.chunk);
    if (p.nparts < 1) p.nparts = 1;
    return p;
}

template <bool ROWS, bool EXACT>
cudaError_t gram_launch(const float *M, int64_t N, int64_t ldm, int r, int rs, float *G,
                        float *G_lo, void *ws, cudaStream_t st) {
    const GramPlan p = plan_gram(N);
    float *part = static_cast<float *>(ws);
    float *part_lo = part + (size_t)p.nparts * rs * rs;
    const int rb = (r + 15) / 16;
    switch (rb) {
#define NMF_GRAM_CASE(RBV)                                                                     \
    case RBV:                                                                                  \
        gram_partial_kernel<RBV, ROWS, EXACT><<<p.nparts, 256, 0, st>>>(M, N, ldm, r, p.chunk,  \
                                                                        part, part_lo, rs);    \
        break;
        NMF_GRAM_CASE(1) NMF_GRAM_CASE(2) NMF_GRAM_CASE(3) NMF_GRAM_CASE(4)
        NMF_GRAM_CASE(5) NMF_GRAM_CASE(6) NMF_GRAM_CASE(7) NMF_GRAM_CASE(8)
#undef NMF_GRAM_CASE
        default: return cudaErrorInvalidValue;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const unsigned rgrid = (unsigned)((rs * rs + 31) / 32);
    if constexpr (EXACT)
        gram_reduce_exact_kernel<<<rgrid, kRedWarps * 32, 0, st>>>(part, part_lo, p.nparts, rs, G,
                                                                   G_lo);
    else
        gram_reduce_kernel<<<rgrid, kRedWarps * 32, 0, st>>>(part, p.nparts, rs, G);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- e(0)
// Per row i of W, Remark 1 in residual form: <w_i, c_i> and <w_i, D w_i - c_i>
// with c = C + C_lo, D = D + D_lo; D w - c evaluated with error-free
// products and sums, both terms accumulated across rows in FP64.
__global__ void __launch_bounds__(256)
err_rows_kernel(int64_t m, int r, int rs, const float *__restrict__ W,
                const float *__restrict__ C, const float *__restrict__ C_lo,
                const float *__restrict__ D, const float *__restrict__ D_lo,
                ErrPartial *__restrict__ part) {
    extern __shared__ float Ds[];   // rs x rs hi, then rs x rs lo
    __shared__ double red[256 / 32];
    for (int e = threadIdx.x; e < rs * rs; e += blockDim.x) {
        Ds[e] = D[e];
        Ds[rs * rs + e] = D_lo[e];
    }
    __syncthreads();
    double cross = 0.0, quad = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float *w = W + i * rs;
        for (int k = 0; k < r; ++k) {
            float hi = -C[i * rs + k], lo = -C_lo[i * rs + k];
            for (int j = 0; j < r; ++j) {
                float p, pe, sum, se;
                two_prod(Ds[k * rs + j], w[j], p, pe);
                two_sum(hi, p, sum, se);
                hi = sum;
                lo += se + pe + Ds[rs * rs + k * rs + j] * w[j];
            }
            cross = fma((double)w[k], (double)C[i * rs + k] + (double)C_lo[i * rs + k], cross);
            quad = fma((double)w[k], (double)hi + (double)lo, quad);
        }
    }
    const double cs = block_sum_d<256>(cross, red);
    const double qs = block_sum_d<256>(quad, red);
    if (threadIdx.x == 0) {
        part[blockIdx.x].cross = cs;
        part[blockIdx.x].quad = qs;
    }
}

// Remark 1 (residual form) of a given pair from the err_rows partials:
// out[0] = e^2 = ||X||^2 - cross + quad (unclamped), out[1] = sqrt(max(0, e^2)).
__global__ void pair_error_kernel(const ErrPartial *__restrict__ part, int nparts,
                                  const double *__restrict__ fro2, double *__restrict__ out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double c = 0.0, q = 0.0;
    for (int p = 0; p < nparts; ++p) {
        c += part[p].cross;
        q += part[p].quad;
    }
    const double e2 = *fro2 - c + q;
    out[0] = e2;
    out[1] = sqrt(e2 > 0.0 ? e2 : 0.0);
}

__global__ void init_state_kernel(const ErrPartial *__restrict__ part, int nparts,
                                  const double *__restrict__ fro2, DevState *__restrict__ s,
                                  double beta0) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double c = 0.0, q = 0.0;
    for (int p = 0; p < nparts; ++p) {
        c += part[p].cross;
        q += part[p].quad;
    }
    const double f = *fro2;
    const double e2 = f - c + q;      // residual form of Remark 1
    const double e = sqrt(e2 > 0.0 ? e2 : 0.0);
    s->fro2 = f;
    s->e_last = e;
    s->e_prev = e;
    s->e_k = e;
    s->beta = beta0;
    s->beta_bar = 1.0;
    s->beta_prev = beta0;
    s->beta_used = beta0;
    s->k = 0;
    s->accepted = 1;
    s->status = isfinite(e2) ? 0 : (int)NMF_ENONFINITE;
}

// ---------------------------------------------------------------- finalize
// W part: q < m*rs, H part: q < r*ldh.  Padded entries are zero everywhere
// and stay zero.
__device__ __forceinline__ void
finalize_body(int64_t nw, int64_t nh, float *__restrict__ W, float *__restrict__ H,
              float *__restrict__ Wy, float *__restrict__ Hy, const float *__restrict__ Wn,
              const float *__restrict__ Hn, const float *__restrict__ Hw,
              const DevState *__restrict__ state, const DevParams &p, int64_t bid, int64_t nblk) {
    const int acc = state->accepted;
    const float beta = (float)state->beta_used;
    const int64_t stride = nblk * blockDim.x;
    for (int64_t q = bid * blockDim.x + threadIdx.x; q < nw + nh; q += stride) {
        if (q < nw) {
            if (acc) {
                const float wold = W[q], wn = Wn[q];
                float wy = fmaf(beta, wn - wold, wn);          // step 11
                if (p.project_w) wy = fmaxf(wy, 0.0f);
                W[q] = wn;                                     // step 19
                Wy[q] = wy;
            } else {
                Wy[q] = W[q];                                  // step 17
            }
        } else {
            const int64_t h = q - nw;
            if (acc) {
                const float hold = H[h], hn = Hn[h];
                float hy;
                if (p.hp == 1) hy = fmaf(beta, hn - hold, hn); // step 13
                else hy = Hw[h];                               // steps 4-9
                H[h] = hn;
                Hy[h] = hy;
            } else {
                Hy[h] = H[h];
            }
        }
    }
}

__global__ void __launch_bounds__(256)
finalize_kernel(int64_t nw, int64_t nh, float *__restrict__ W, float *__restrict__ H,
                float *__restrict__ Wy, float *__restrict__ Hy, const float *__restrict__ Wn,
                const float *__restrict__ Hn, const float *__restrict__ Hw,
                const DevState *__restrict__ state, DevParams p) {
    finalize_body(nw, nh, W, H, Wy, Hy, Wn, Hn, Hw, state, p, blockIdx.x, gridDim.x);
}
__global__ void __launch_bounds__(256)
finalize_grouped(const FinalizeItem *__restrict__ items, const int64_t *__restrict__ begin,
                 int nitems) {
    int64_t local;
    const int i = group_item(begin, nitems, local);
    const FinalizeItem &it = items[i];
    finalize_body(it.nw, it.nh, it.W, it.H, it.Wy, it.Hy, it.Wn, it.Hn, it.Hw, it.state, it.p,
                  local, __ldg(begin + i + 1) - __ldg(begin + i));
}

__global__ void nonfinite_kernel(const float *__restrict__ v, int64_t count, int *flag) {
    int bad = 0;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < count;
         q += (int64_t)gridDim.x * blockDim.x)
        bad |= !isfinite(v[q]);
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flag, 1);
}

}  // namespace

size_t fro2_ws_bytes(int64_t) { return sizeof(double) * kRedBlocks; }

cudaError_t launch_fro2(const float *vals, int64_t rows, int64_t cols, int64_t ld, double *out,
                        void *ws, cudaStream_t st) {
    double *part = static_cast<double *>(ws);
    fro2_partial_kernel<<<kRedBlocks, kRedThreads, 0, st>>>(vals, rows, cols, ld, part);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    sum_partials_kernel<<<1, kRedThreads, 0, st>>>(part, kRedBlocks, out);
    return cudaGetLastError();
}

size_t gram_ws_bytes(int64_t N, int rs) {
    const GramPlan p = plan_gram(N);
    return 2 * sizeof(float) * (size_t)p.nparts * rs * rs;
}

cudaError_t launch_gram_rows(const float *M, int64_t N, int64_t ldm, int r, int rs, float *G,
                             void *ws, cudaStream_t st) {
    return gram_launch<true, false>(M, N, ldm, r, rs, G, nullptr, ws, st);
}

cudaError_t launch_gram_rows_exact(const float *M, int64_t N, int64_t ldm, int r, int rs,
                                   float *G, float *G_lo, void *ws, cudaStream_t st) {
    return gram_launch<true, true>(M, N, ldm, r, rs, G, G_lo, ws, st);
}

cudaError_t launch_gram_cols(const float *M, int64_t N, int64_t ldm, int r, int rs, float *G,
                             float *G_lo, void *ws, cudaStream_t st) {
    return gram_launch<false, true>(M, N, ldm, r, rs, G, G_lo, ws, st);
}

int err_rows_num_ctas(int64_t m) {
    int64_t b = (m + 255) / 256;
    if (b > 2 * kNumSMs) b = 2 * kNumSMs;
    return (int)(b < 1 ? 1 : b);
}

cudaError_t launch_err_rows(int64_t m, int r, int rs, const float *W, const float *C,
                            const float *C_lo, const float *D, const float *D_lo,
                            ErrPartial *part, cudaStream_t st) {
    const size_t smem = 2 * sizeof(float) * (size_t)rs * rs;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(err_rows_kernel,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
    }
    err_rows_kernel<<<err_rows_num_ctas(m), 256, smem, st>>>(m, r, rs, W, C, C_lo, D, D_lo, part);
    return cudaGetLastError();
}

cudaError_t launch_init_state(int64_t m, int r, int rs, const float *W, const float *C,
                              const float *C_lo, const float *D, const float *D_lo,
                              const double *fro2, DevState *state, double beta0,
                              ErrPartial *partials, cudaStream_t st) {
    cudaError_t e = launch_err_rows(m, r, rs, W, C, C_lo, D, D_lo, partials, st);
    if (e != cudaSuccess) return e;
    init_state_kernel<<<1, 32, 0, st>>>(partials, err_rows_num_ctas(m), fro2, state, beta0);
    return cudaGetLastError();
}

cudaError_t launch_pair_error(int64_t m, const double *fro2, const ErrPartial *partials,
                              double *out, cudaStream_t st) {
    pair_error_kernel<<<1, 32, 0, st>>>(partials, err_rows_num_ctas(m), fro2, out);
    return cudaGetLastError();
}

cudaError_t launch_finalize(int64_t m, int rs, int r, int64_t ldh, float *W, float *H,
                            float *Wy, float *Hy, const float *Wn, const float *Hn,
                            const float *Hw, const DevState *state, DevParams p,
                            cudaStream_t st) {
    const int64_t nw = m * rs, nh = (int64_t)r * ldh;
    int64_t blocks = (nw + nh + 255) / 256;
    if (blocks > 8 * kNumSMs) blocks = 8 * kNumSMs;
    finalize_kernel<<<(unsigned)blocks, 256, 0, st>>>(nw, nh, W, H, Wy, Hy, Wn, Hn, Hw, state, p);
    return cudaGetLastError();
}

cudaError_t launch_nonfinite_scan(const float *v, int64_t count, int *flag, cudaStream_t st) {
    int64_t blocks = (count + 255) / 256;
    if (blocks > 4 * kNumSMs) blocks = 4 * kNumSMs;
    if (blocks < 1) blocks = 1;
    nonfinite_kernel<<<(unsigned)blocks, 256, 0, st>>>(v, count, flag);
    return cudaGetLastError();
}


// ------------------------------------------------------------ grouped launches
// (The Gram of W in FP32 and the error-free Gram of H: the variants of the
// batched HALS iteration.)
int gram_group_key(int r, bool rows, bool exact) {
    return ((r + 15) / 16) * 4 + (rows ? 2 : 0) + (exact ? 1 : 0);
}

void plan_gram_item(const float *M, int64_t N, int64_t ldm, int r, int rs, float *G,
                    float *G_lo, void *ws, GramItem *it, int64_t *ctas_partial,
                    int64_t *ctas_reduce) {
    const GramPlan p = plan_gram(N);
    float *part = static_cast<float *>(ws);
    *it = GramItem{M, N, ldm, r, rs, p.chunk, part, part + (size_t)p.nparts * rs * rs, p.nparts,
                   G, G_lo};
    *ctas_partial = p.nparts;
    *ctas_reduce = (rs * rs + 31) / 32;
}

cudaError_t launch_gram_partial_grouped(int key, const GramItem *items, const int64_t *begin,
                                        int nitems, int64_t ctas, cudaStream_t st) {
    if (nitems < 1 || ctas < 1) return cudaSuccess;
    const int rb = key / 4;
    const bool rows = (key & 2) != 0, exact = (key & 1) != 0;
    switch (rb) {
#define NMF_GRAM_GROUPED(RBV)                                                                  \
    case RBV:                                                                                  \
        if (rows && !exact)                                                                    \
            gram_partial_grouped<RBV, true, false><<<(unsigned)ctas, 256, 0, st>>>(items, begin, \
                                                                                  nitems);     \
        else if (!rows && exact)                                                               \
            gram_partial_grouped<RBV, false, true><<<(unsigned)ctas, 256, 0, st>>>(items, begin, \
                                                                                  nitems);     \
        else                                                                                   \
            return cudaErrorInvalidValue;                                                      \
        return cudaGetLastError();
        NMF_GRAM_GROUPED(1) NMF_GRAM_GROUPED(2) NMF_GRAM_GROUPED(3) NMF_GRAM_GROUPED(4)
        NMF_GRAM_GROUPED(5) NMF_GRAM_GROUPED(6) NMF_GRAM_GROUPED(7) NMF_GRAM_GROUPED(8)
#undef NMF_GRAM_GROUPED
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_gram_reduce_grouped(bool exact, const GramItem *items, const int64_t *begin,
                                       int nitems, int64_t ctas, cudaStream_t st) {
    if (nitems < 1 || ctas < 1) return cudaSuccess;
    if (exact)
        gram_reduce_grouped<true><<<(unsigned)ctas, kRedWarps * 32, 0, st>>>(items, begin, nitems);
    else
        gram_reduce_grouped<false><<<(unsigned)ctas, kRedWarps * 32, 0, st>>>(items, begin, nitems);
    return cudaGetLastError();
}

void plan_finalize_item(int64_t m, int rs, int r, int64_t ldh, float *W, float *H, float *Wy,
                        float *Hy, const float *Wn, const float *Hn, const float *Hw,
                        const DevState *state, DevParams p, FinalizeItem *it, int64_t *ctas) {
    // Elementwise, so any grid gives the same result: eight entries per
    // thread (the many small instances of a batch need no more CTAs).
    const int64_t nw = m * rs, nh = (int64_t)r * ldh;
    int64_t blocks = (nw + nh + 8 * 256 - 1) / (8 * 256);
    if (blocks > 8 * kNumSMs) blocks = 8 * kNumSMs;
    *it = FinalizeItem{nw, nh, W, H, Wy, Hy, Wn, Hn, Hw, state, p};
    *ctas = blocks;
}

cudaError_t launch_finalize_grouped(const FinalizeItem *items, const int64_t *begin, int nitems,
                                    int64_t ctas, cudaStream_t st) {
    if (nitems < 1 || ctas < 1) return cudaSuccess;
    finalize_grouped<<<(unsigned)ctas, 256, 0, st>>>(items, begin, nitems);
    return cudaGetLastError();
}

}  // namespace nmfg
