// products.cu -- the two X products of every outer iteration, FP32 on CUDA
// cores:
//   A = W_y^T X   (r x n), the W(:,k)^T X term of the HALS closed form (Sec. 1)
//   C = X H_y^T   (m x r), the X H^T term of Remark 1 / the W-update
// Both stream X once.  X is m x ldx row-major with ldx a multiple of 8 (the
// library pads its copy with zeros), W/C are m x rs, H/A are r x ldh.
//
// Tiles are staged global -> shared with cp.async (16-byte, L1-bypassing)
// through a 3-stage ring.  Sums are compensated: every 32-deep stage is
// accumulated in FP32, and the stage sums (and the split-K partials) are
// combined with Kahan's correction, which keeps the products within a few
// units in the last place of the exact value for the sum lengths met here.  A uses a deterministic split-K over the rows of
// X: every split writes its partial tile, and the last split of a column
// tile to finish (atomic ticket) adds the partials in split order.
#include <cuda_runtime.h>

#include "common.cuh"

namespace nmfg {
namespace {

constexpr int kThreads = 128;
constexpr int kStages = 3;
constexpr int BK = 32;          // reduction depth per stage
constexpr int PADK = BK + 4;    // smem row stride (floats), keeps 16-byte rows

__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gsrc, bool pred) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    const int src_bytes = pred ? 16 : 0;   // 0 -> zero fill
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(gsrc),
                 "r"(src_bytes));
}
// The same for X, which each product reads exactly once: marked to leave L2
// first, so that streaming it does not push out the factors and the split
// partials that are read again.
__device__ __forceinline__ uint64_t evict_first_policy() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
__device__ __forceinline__ void cp_async16_stream(void *smem_dst, const void *gsrc, bool pred,
                                                  uint64_t pol) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    const int src_bytes = pred ? 16 : 0;   // 0 -> zero fill
    asm volatile("cp.async.cg.shared.global.L2::cache_hint [%0], [%1], 16, %2, %3;\n" ::"r"(d),
                 "l"(gsrc), "r"(src_bytes), "l"(pol));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

// Kahan's compensated addition: (sum, c) absorbs v; sum - c is the result.
__device__ __forceinline__ void kahan_add(float &sum, float &c, float v) {
    const float y = v - c;
    const float t = sum + y;
    c = (t - sum) - y;
    sum = t;
}

// ---------------------------------------------------------------------------
// C = X H^T.  CTA: BM = 16*TM rows of X, all R = 8*TR columns of C.
// Thread (tx in 0..7, ty in 0..15) owns rows ty + 16a and columns tx + 8b.
// ---------------------------------------------------------------------------
template <int TM, int TR>
__device__ __forceinline__ void
xht_body(const float *__restrict__ X, int64_t m, int64_t ldx, int r,
         const float *__restrict__ H, int64_t ldh, float *__restrict__ C,
         float *__restrict__ C_lo, int rs, int64_t cols_per_split,
         float *__restrict__ part, unsigned int *__restrict__ tickets,
         int64_t tile, int split, int nsplit) {
    constexpr int BM = 16 * TM;
    constexpr int R = 8 * TR;
    extern __shared__ __align__(16) float sm[];
    float *Xs = sm;                                   // [kStages][BM][PADK]
    float *Hs = sm + kStages * BM * PADK;             // [kStages][R][PADK]
    __shared__ bool am_last;

    const int tid = threadIdx.x;
    const int tx = tid % 8, ty = tid / 8;
    const int64_t row0 = tile * BM;
    const int64_t kbeg = (int64_t)split * cols_per_split;
    const int64_t kend = min(ldx, kbeg + cols_per_split);
    const int64_t nk = kend > kbeg ? (kend - kbeg + BK - 1) / BK : 0;

    // Each thread always copies the same 16-byte column c4 of rows
    // lr, lr + 16, ... of both tiles (kThreads is a multiple of BK/4), so the
    // addresses are formed once and advance by BK per stage.
    constexpr int kRowsPerPass = kThreads / (BK / 4);
    const int lr = tid / (BK / 4), c4 = tid % (BK / 4);
    const float *xg = X + (row0 + lr) * ldx + kbeg + c4 * 4;
    const uint64_t pol = evict_first_policy();
    const float *hg = H + (int64_t)lr * ldh + kbeg + c4 * 4;
    auto load_stage = [&](int stage, int64_t kt) {
        const int64_t koff = kt * BK;
        const bool colok = kbeg + koff + c4 * 4 < kend;
        float *xs = Xs + stage * BM * PADK + lr * PADK + c4 * 4;
#pragma unroll
        for (int j = 0; j < BM / kRowsPerPass; ++j) {
            const bool ok = colok && row0 + lr + j * kRowsPerPass < m;
            cp_async16_stream(xs + j * kRowsPerPass * PADK,
                              ok ? xg + (int64_t)j * kRowsPerPass * ldx + koff : X, ok, pol);
        }
        float *hs = Hs + stage * R * PADK + lr * PADK + c4 * 4;
#pragma unroll
        for (int j = 0; j < (R + kRowsPerPass - 1) / kRowsPerPass; ++j) {
            const int kk = lr + j * kRowsPerPass;
            if (kk < R) {
                const bool ok = colok && kk < r;
                cp_async16(hs + j * kRowsPerPass * PADK,
                           ok ? hg + (int64_t)j * kRowsPerPass * ldh + koff : H, ok);
            }
        }
    };

    // Compensated accumulation: each 32-deep stage is summed into `blk`, and
    // the stage sums are added into (acc, comp) with Kahan's correction.
    float acc[TM][TR], comp[TM][TR];
#pragma unroll
    for (int a = 0; a < TM; ++a)
#pragma unroll
        for (int b = 0; b < TR; ++b) acc[a][b] = comp[a][b] = 0.0f;

#pragma unroll
    for (int s = 0; s < kStages - 1; ++s) {
        if (s < nk) load_stage(s, s);
        cp_async_commit();
    }

    for (int64_t kt = 0; kt < nk; ++kt) {
        cp_async_wait<kStages - 2>();
        __syncthreads();
        const int64_t nxt = kt + kStages - 1;
        if (nxt < nk) load_stage((int)(nxt % kStages), nxt);
        cp_async_commit();

        const float *xs = Xs + (kt % kStages) * BM * PADK;
        const float *hs = Hs + (kt % kStages) * R * PADK;
        float blk[TM][TR];
#pragma unroll
        for (int a = 0; a < TM; ++a)
#pragma unroll
            for (int b = 0; b < TR; ++b) blk[a][b] = 0.0f;
#pragma unroll
        for (int kk = 0; kk < BK; kk += 4) {
            float4 xv[TM], hv[TR];
#pragma unroll
            for (int a = 0; a < TM; ++a)
                xv[a] = *reinterpret_cast<const float4 *>(xs + (ty + 16 * a) * PADK + kk);
#pragma unroll
            for (int b = 0; b < TR; ++b)
                hv[b] = *reinterpret_cast<const float4 *>(hs + (tx + 8 * b) * PADK + kk);
#pragma unroll
            for (int a = 0; a < TM; ++a)
#pragma unroll
                for (int b = 0; b < TR; ++b) {
                    blk[a][b] = fmaf(xv[a].x, hv[b].x, blk[a][b]);
                    blk[a][b] = fmaf(xv[a].y, hv[b].y, blk[a][b]);
                    blk[a][b] = fmaf(xv[a].z, hv[b].z, blk[a][b]);
                    blk[a][b] = fmaf(xv[a].w, hv[b].w, blk[a][b]);
                }
        }
#pragma unroll
        for (int a = 0; a < TM; ++a)
#pragma unroll
            for (int b = 0; b < TR; ++b) kahan_add(acc[a][b], comp[a][b], blk[a][b]);
    }
    cp_async_wait<0>();

    // The compensated sum is acc - comp; C keeps its FP32 rounding and C_lo
    // the remainder (the Remark 1 error term <W, C> uses both).
    if (nsplit == 1) {
#pragma unroll
        for (int a = 0; a < TM; ++a) {
            const int64_t row = row0 + ty + 16 * a;
            if (row >= m) continue;
#pragma unroll
            for (int b = 0; b < TR; ++b) {
                const int col = tx + 8 * b;
                if (col < rs) {
                    const float hi = acc[a][b] - comp[a][b];
                    C[row * rs + col] = hi;
                    C_lo[row * rs + col] = (acc[a][b] - hi) - comp[a][b];
                }
            }
        }
        return;
    }
    // Split-K over the columns of X: partial tiles (hi, lo), summed in split
    // order by the last split of the row tile to finish.
    float *my = part + (tile * nsplit + split) * (2 * BM * R);
#pragma unroll
    for (int a = 0; a < TM; ++a)
#pragma unroll
        for (int b = 0; b < TR; ++b) {
            const float hi = acc[a][b] - comp[a][b];
            my[(ty + 16 * a) * R + tx + 8 * b] = hi;
            my[BM * R + (ty + 16 * a) * R + tx + 8 * b] = (acc[a][b] - hi) - comp[a][b];
        }
    __threadfence();
    __syncthreads();
    if (tid == 0) {
        const unsigned int tk = atomicAdd(tickets + tile, 1u);
        am_last = (tk == (unsigned)nsplit - 1);
    }
    __syncthreads();
    if (!am_last) return;
    __threadfence();
    // Each thread sums its TM*TR elements over the splits in split order,
    // all of one split's loads in flight at once.
    const float *base = part + tile * nsplit * (2 * BM * R);
    constexpr int J = BM * R / kThreads;
    static_assert(J * kThreads == BM * R, "tile must divide among the threads");
    float fh[J], fl[J];
#pragma unroll
    for (int j = 0; j < J; ++j) fh[j] = fl[j] = 0.0f;
    for (int q = 0; q < nsplit; ++q) {
        const float *ph = base + (int64_t)q * 2 * BM * R;
        float vh[J], vl[J];
#pragma unroll
        for (int j = 0; j < J; ++j) {
            vh[j] = __ldcg(ph + tid + j * kThreads);
            vl[j] = __ldcg(ph + BM * R + tid + j * kThreads);
        }
#pragma unroll
        for (int j = 0; j < J; ++j) {
            const float s = fh[j] + vh[j], bb = s - fh[j];
            fl[j] += (fh[j] - (s - bb)) + (vh[j] - bb) + vl[j];
            fh[j] = s;
        }
    }
#pragma unroll
    for (int j = 0; j < J; ++j) {
        const int e = tid + j * kThreads;
        const int64_t row = row0 + e / R;
        const int col = e % R;
        if (row < m && col < rs) {
            const float c = fh[j] + fl[j];
            C[row * rs + col] = c;
            C_lo[row * rs + col] = (fh[j] - c) + fl[j];
        }
    }
    if (tid == 0) tickets[tile] = 0u;
}

// ---------------------------------------------------------------------------
// A = W^T X.  CTA: BN = 128 columns of X, all R = rs rows of A, rows
// [i_begin, i_end) of X (a split of the reduction).  4R threads: thread
// (g, tx), g < R/4, tx < 16, owns the rows 4g..4g+3 of A and the columns
// 4tx..4tx+3 and 64+4tx..64+4tx+3 of the tile, so each X row of the stage
// costs it three 16-byte shared loads for 32 FMAs.
// ---------------------------------------------------------------------------
constexpr int BN = 128;
constexpr int PADN = BN + 4;

template <int R>
__device__ __forceinline__ void
wtx_body(const float *__restrict__ X, int64_t m, int64_t ldx, int r,
         const float *__restrict__ W, float *__restrict__ A, int64_t lda,
         int64_t rows_per_split, float *__restrict__ part,
         unsigned int *__restrict__ tickets, int64_t tile, int split, int nsplit) {
    constexpr int NT = 4 * R;
    constexpr int PADR = R + 4;
    extern __shared__ __align__(16) float sm[];
    float *Xs = sm;                                   // [kStages][BK][PADN]
    float *Ws = sm + kStages * BK * PADN;             // [kStages][BK][PADR]
    __shared__ bool am_last;

    const int tid = threadIdx.x;
    const int tx = tid % 16, g = tid / 16;
    const int64_t col0 = tile * BN;
    const int64_t i_begin = (int64_t)split * rows_per_split;
    const int64_t i_end = min(m, i_begin + rows_per_split);
    const int64_t nk = i_end > i_begin ? (i_end - i_begin + BK - 1) / BK : 0;
    const uint64_t pol = evict_first_policy();

    auto load_stage = [&](int stage, int64_t kt) {
        const int64_t i0 = i_begin + kt * BK;
        float *xs = Xs + stage * BK * PADN;
        for (int idx = tid; idx < BK * (BN / 4); idx += NT) {
            const int ii = idx / (BN / 4), c4 = idx % (BN / 4);
            const int64_t grow = i0 + ii, gcol = col0 + c4 * 4;
            const bool ok = grow < i_end && gcol < ldx;
            cp_async16_stream(xs + ii * PADN + c4 * 4, ok ? X + grow * ldx + gcol : X, ok, pol);
        }
        float *ws = Ws + stage * BK * PADR;
        for (int idx = tid; idx < BK * (R / 4); idx += NT) {
            const int ii = idx / (R / 4), c4 = idx % (R / 4);
            const int64_t grow = i0 + ii;
            const bool ok = grow < i_end;
            cp_async16(ws + ii * PADR + c4 * 4, ok ? W + grow * R + c4 * 4 : W, ok);
        }
    };

    // Compensated accumulation (see the file header).
    float acc[4][8], comp[4][8];
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
        for (int c = 0; c < 8; ++c) acc[b][c] = comp[b][c] = 0.0f;

#pragma unroll
    for (int s = 0; s < kStages - 1; ++s) {
        if (s < nk) load_stage(s, s);
        cp_async_commit();
    }
    for (int64_t kt = 0; kt < nk; ++kt) {
        cp_async_wait<kStages - 2>();
        __syncthreads();
        const int64_t nxt = kt + kStages - 1;
        if (nxt < nk) load_stage((int)(nxt % kStages), nxt);
        cp_async_commit();

        const float *xs = Xs + (kt % kStages) * BK * PADN;
        const float *ws = Ws + (kt % kStages) * BK * PADR;
        float blk[4][8];
#pragma unroll
        for (int b = 0; b < 4; ++b)
#pragma unroll
            for (int c = 0; c < 8; ++c) blk[b][c] = 0.0f;
        // Paired FP32 FMAs: columns (c, c + 1) of a row of A in one
        // instruction, each the same IEEE FMA as a scalar one.
#pragma unroll 4
        for (int ii = 0; ii < BK; ++ii) {
            const float4 w = *reinterpret_cast<const float4 *>(ws + ii * PADR + 4 * g);
            const float4 x0 = *reinterpret_cast<const float4 *>(xs + ii * PADN + 4 * tx);
            const float4 x1 = *reinterpret_cast<const float4 *>(xs + ii * PADN + 64 + 4 * tx);
            const float wv[4] = {w.x, w.y, w.z, w.w};
            const float2 xv[4] = {make_float2(x0.x, x0.y), make_float2(x0.z, x0.w),
                                  make_float2(x1.x, x1.y), make_float2(x1.z, x1.w)};
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const float2 wb = make_float2(wv[b], wv[b]);
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const float2 t = __ffma2_rn(wb, xv[c],
                                                make_float2(blk[b][2 * c], blk[b][2 * c + 1]));
                    blk[b][2 * c] = t.x;
                    blk[b][2 * c + 1] = t.y;
                }
            }
        }
#pragma unroll
        for (int b = 0; b < 4; ++b)
#pragma unroll
            for (int c = 0; c < 8; ++c) kahan_add(acc[b][c], comp[b][c], blk[b][c]);
    }
    cp_async_wait<0>();
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
        for (int c = 0; c < 8; ++c) acc[b][c] -= comp[b][c];

    auto col_of = [&](int c) -> int64_t { return col0 + (c < 4 ? 4 * tx + c : 64 + 4 * tx + c - 4); };
    if (nsplit == 1) {
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int k = 4 * g + b;
            if (k >= r) continue;
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const int64_t j = col_of(c);
                if (j < lda) A[(int64_t)k * lda + j] = acc[b][c];
            }
        }
        return;
    }

    // Split-K: write this split's partial tile, then the last split of the
    // column tile sums the partials in split order.
    float *my = part + (tile * nsplit + split) * (R * BN);
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        float *rowp = my + (4 * g + b) * BN;
        *reinterpret_cast<float4 *>(rowp + 4 * tx) =
            make_float4(acc[b][0], acc[b][1], acc[b][2], acc[b][3]);
        *reinterpret_cast<float4 *>(rowp + 64 + 4 * tx) =
            make_float4(acc[b][4], acc[b][5], acc[b][6], acc[b][7]);
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) {
        const unsigned int t = atomicAdd(tickets + tile, 1u);
        am_last = (t == (unsigned)nsplit - 1);
    }
    __syncthreads();
    if (!am_last) return;
    __threadfence();
    // Each thread sums its float4 words over the splits in split order (Kahan),
    // all of one split's loads in flight at once.
    const float *base = part + tile * nsplit * (R * BN);
    constexpr int J = R * BN / (NT * 4);
    static_assert(J * NT * 4 == R * BN, "tile must divide among the threads");
    float4 fs[J], fc[J];
#pragma unroll
    for (int j = 0; j < J; ++j) fs[j] = fc[j] = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int q = 0; q < nsplit; ++q) {
        const float4 *pq = reinterpret_cast<const float4 *>(base + (int64_t)q * R * BN);
        float4 v[J];
#pragma unroll
        for (int j = 0; j < J; ++j) v[j] = __ldcg(pq + tid + j * NT);
#pragma unroll
        for (int j = 0; j < J; ++j) {
            kahan_add(fs[j].x, fc[j].x, v[j].x);
            kahan_add(fs[j].y, fc[j].y, v[j].y);
            kahan_add(fs[j].z, fc[j].z, v[j].z);
            kahan_add(fs[j].w, fc[j].w, v[j].w);
        }
    }
#pragma unroll
    for (int j = 0; j < J; ++j) {
        const int e = (tid + j * NT) * 4;
        const int k = e / BN;
        const int64_t col = col0 + e % BN;
        if (k < r) {
            const float vv[4] = {fs[j].x - fc[j].x, fs[j].y - fc[j].y, fs[j].z - fc[j].z,
                                 fs[j].w - fc[j].w};
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (col + q < lda) A[(int64_t)k * lda + col + q] = vv[q];
        }
    }
    if (tid == 0) tickets[tile] = 0u;
}

// Single launches: tile = blockIdx.x, split = blockIdx.y.  Grouped launches:
// the item's CTAs in tile-major order of its own (tiles x nsplit) grid.
template <int TM, int TR>
__global__ void __launch_bounds__(kThreads)
xht_f32_kernel(const float *__restrict__ X, int64_t m, int64_t ldx, int r,
               const float *__restrict__ H, int64_t ldh, float *__restrict__ C,
               float *__restrict__ C_lo, int rs, int64_t cols_per_split,
               float *__restrict__ part, unsigned int *__restrict__ tickets) {
    xht_body<TM, TR>(X, m, ldx, r, H, ldh, C, C_lo, rs, cols_per_split, part, tickets,
                     blockIdx.x, blockIdx.y, gridDim.y);
}
template <int TM, int TR>
__global__ void __launch_bounds__(kThreads)
xht_f32_grouped(const XhtItem *__restrict__ items, const int64_t *__restrict__ begin,
                int nitems) {
    int64_t local;
    const XhtItem &it = items[group_item(begin, nitems, local)];
    xht_body<TM, TR>(it.X, it.m, it.ldx, it.r, it.H, it.ldh, it.C, it.C_lo, it.rs,
                     it.cols_per_split, it.part, it.tickets, local % it.tiles,
                     (int)(local / it.tiles), it.nsplit);
}
template <int R>
__global__ void __launch_bounds__(4 * R)
wtx_f32_kernel(const float *__restrict__ X, int64_t m, int64_t ldx, int r,
               const float *__restrict__ W, float *__restrict__ A, int64_t lda,
               int64_t rows_per_split, float *__restrict__ part,
               unsigned int *__restrict__ tickets) {
    wtx_body<R>(X, m, ldx, r, W, A, lda, rows_per_split, part, tickets, blockIdx.x, blockIdx.y,
                gridDim.y);
}
template <int R>
__global__ void __launch_bounds__(4 * R)
wtx_f32_grouped(const WtxItem *__restrict__ items, const int64_t *__restrict__ begin,
                int nitems) {
    int64_t local;
    const WtxItem &it = items[group_item(begin, nitems, local)];
    wtx_body<R>(it.X, it.m, it.ldx, it.r, it.W, it.A, it.lda, it.rows_per_split, it.part,
                it.tickets, local % it.tiles, (int)(local / it.tiles), it.nsplit);
}

// Splits of the reduction for a grid of tiles x nsplit CTAs of which
// `per_sm` fit on an SM at once: the count whose waves fill the GPU best
// (one CTA's time per SM beyond an even share is a tail), preferring fewer
// splits unless more fill the waves by over 2 points.
int balanced_splits(int64_t tiles, int per_sm, int64_t max_split) {
    const int64_t slots = (int64_t)kNumSMs * (per_sm > 0 ? per_sm : 1);
    int best = 1;
    double best_eff = 0.0;
    for (int64_t ns = 1; ns <= max_split; ++ns) {
        const int64_t total = tiles * ns;
        const int64_t waves = (total + slots - 1) / slots;
        const double eff = (double)total / (double)(waves * slots);
        if (eff > best_eff + 0.02) {
            best_eff = eff;
            best = (int)ns;
        }
    }
    return best;
}

template <typename K>
int resident_ctas(K kern, int threads, size_t smem) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, threads, smem) != cudaSuccess) n = 1;
    return n > 0 ? n : 1;
}

constexpr int kMaxWtxSplits = 64;
constexpr int kMaxXhtSplits = 16;

template <int R>
constexpr size_t wtx_smem() {
    return sizeof(float) * (size_t)kStages * BK * (PADN + R + 4);
}
template <int TM, int TR>
constexpr size_t xht_smem() {
    return sizeof(float) * (size_t)kStages * (16 * TM + 8 * TR) * PADK;
}

// The grid of a product: column (row) tiles x splits of the reduction,
// chosen from the CTAs the occupancy calculator fits on an SM.
struct SplitPlan {
    int64_t tiles;
    int nsplit;
    int64_t per_split;      // rows (A) or columns (C) of X per split
};

template <int R>
cudaError_t wtx_prepare(SplitPlan *sp, int64_t m, int64_t lda) {
    const size_t smem = wtx_smem<R>();
    cudaError_t e = cudaFuncSetAttribute(wtx_f32_kernel<R>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(wtx_f32_grouped<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
    if (e != cudaSuccess) return e;
    static const int per_sm = resident_ctas(wtx_f32_kernel<R>, 4 * R, smem);
    sp->tiles = (lda + BN - 1) / BN;
    int64_t max_split = (m + 8 * BK - 1) / (8 * BK);              // >= 256 rows per split
    if (max_split > kMaxWtxSplits) max_split = kMaxWtxSplits;
    const int want = balanced_splits(sp->tiles, per_sm, max_split);
    sp->per_split = ((m + want - 1) / want + BK - 1) / BK * BK;
    sp->nsplit = (int)((m + sp->per_split - 1) / sp->per_split);
    return cudaSuccess;
}

template <int TM, int TR>
cudaError_t xht_prepare(SplitPlan *sp, int64_t m, int64_t ldx) {
    constexpr int BM = 16 * TM;
    const size_t smem = xht_smem<TM, TR>();
    cudaError_t e = cudaFuncSetAttribute(xht_f32_kernel<TM, TR>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(xht_f32_grouped<TM, TR>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    static const int per_sm = resident_ctas(xht_f32_kernel<TM, TR>, kThreads, smem);
    sp->tiles = (m + BM - 1) / BM;
    int64_t max_split = (ldx + 8 * BK - 1) / (8 * BK);            // >= 256 columns per split
    if (max_split > kMaxXhtSplits) max_split = kMaxXhtSplits;
    const int want = balanced_splits(sp->tiles, per_sm, max_split);
    sp->per_split = ((ldx + want - 1) / want + BK - 1) / BK * BK;
    sp->nsplit = (int)((ldx + sp->per_split - 1) / sp->per_split);
    return cudaSuccess;
}

template <int R>
cudaError_t wtx_launch(const float *X, int64_t m, int64_t ldx, int r, const float *W, float *A,
                       int64_t lda, float *part, unsigned int *tickets, cudaStream_t st) {
    SplitPlan sp;
    cudaError_t e = wtx_prepare<R>(&sp, m, lda);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)sp.tiles, (unsigned)sp.nsplit);
    wtx_f32_kernel<R><<<grid, 4 * R, wtx_smem<R>(), st>>>(X, m, ldx, r, W, A, lda, sp.per_split,
                                                          part, tickets);
    return cudaGetLastError();
}

template <int TM, int TR>
cudaError_t xht_launch(const float *X, int64_t m, int64_t ldx, int r, const float *H,
                       int64_t ldh, float *C, float *C_lo, int rs, float *part,
                       unsigned int *tickets, cudaStream_t st) {
    SplitPlan sp;
    cudaError_t e = xht_prepare<TM, TR>(&sp, m, ldx);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)sp.tiles, (unsigned)sp.nsplit);
    xht_f32_kernel<TM, TR><<<grid, kThreads, xht_smem<TM, TR>(), st>>>(
        X, m, ldx, r, H, ldh, C, C_lo, rs, sp.per_split, part, tickets);
    return cudaGetLastError();
}

// Row-tile height of C = X H^T: 64-row tiles once they cover every SM
// (32-row tiles for r > 72, where the 64-row tile spills).  The split of n
// is chosen at launch (balanced_splits); the workspace holds the largest.
bool xht_big(int64_t m, int r) { return m >= (int64_t)kNumSMs * 64 && r <= 72; }

}  // namespace

size_t wtx_ws_bytes(int64_t m, int64_t lda, int r) {
    (void)m;
    const int R = 8 * ((r + 7) / 8);
    return sizeof(float) * (size_t)((lda + BN - 1) / BN) * kMaxWtxSplits * R * BN;
}

int64_t wtx_num_tickets(int64_t lda) { return (lda + BN - 1) / BN; }

cudaError_t launch_wtx_f32(const float *X, int64_t m, int64_t lda, int64_t ldx, int r,
                           const float *W, int rs, float *A, void *ws, unsigned int *tickets,
                           cudaStream_t st) {
    float *part = static_cast<float *>(ws);
    switch (rs) {
#define NMF_WTX_CASE(RV)                                                                      \
    case RV:                                                                                  \
        return wtx_launch<RV>(X, m, ldx, r, W, A, lda, part, tickets, st);
        NMF_WTX_CASE(8) NMF_WTX_CASE(16) NMF_WTX_CASE(24) NMF_WTX_CASE(32)
        NMF_WTX_CASE(40) NMF_WTX_CASE(48) NMF_WTX_CASE(56) NMF_WTX_CASE(64)
        NMF_WTX_CASE(72) NMF_WTX_CASE(80) NMF_WTX_CASE(88) NMF_WTX_CASE(96)
        NMF_WTX_CASE(104) NMF_WTX_CASE(112) NMF_WTX_CASE(120) NMF_WTX_CASE(128)
#undef NMF_WTX_CASE
        default: return cudaErrorInvalidValue;
    }
}

size_t xht_ws_bytes(int64_t m, int64_t ldx, int r) {
    (void)ldx;
    const int64_t bm = xht_big(m, r) ? 64 : 32;
    return 2 * sizeof(float) * (size_t)((m + bm - 1) / bm) * kMaxXhtSplits * bm *
           (8 * ((r + 7) / 8));
}

int64_t xht_num_tickets(int64_t m) { return (m + 31) / 32; }

cudaError_t launch_xht_f32(const float *X, int64_t m, int64_t ldx, int r, const float *H,
                           int64_t ldh, float *C, float *C_lo, int rs, void *ws,
                           unsigned int *tickets, cudaStream_t st) {
    const bool big = xht_big(m, r);
    float *part = static_cast<float *>(ws);
    switch ((r + 7) / 8) {
#define NMF_XHT_CASE(TRV)                                                                      \
    case TRV:                                                                                  \
        return big ? xht_launch<4, TRV>(X, m, ldx, r, H, ldh, C, C_lo, rs, part, tickets, st)   \
                   : xht_launch<2, TRV>(X, m, ldx, r, H, ldh, C, C_lo, rs, part, tickets, st);
        NMF_XHT_CASE(1) NMF_XHT_CASE(2) NMF_XHT_CASE(3) NMF_XHT_CASE(4)
        NMF_XHT_CASE(5) NMF_XHT_CASE(6) NMF_XHT_CASE(7) NMF_XHT_CASE(8)
        NMF_XHT_CASE(9) NMF_XHT_CASE(10) NMF_XHT_CASE(11) NMF_XHT_CASE(12)
        NMF_XHT_CASE(13) NMF_XHT_CASE(14) NMF_XHT_CASE(15) NMF_XHT_CASE(16)
#undef NMF_XHT_CASE
        default: return cudaErrorInvalidValue;
    }
}


// ------------------------------------------------------------ grouped launches
// Key of a product variant: A = W^T X by rs; C = X H^T by (tile height, rs / 8).
int wtx_group_key(int rs) { return rs; }
int xht_group_key(int64_t m, int r) { return (xht_big(m, r) ? 4 : 2) * 32 + (r + 7) / 8; }

cudaError_t plan_wtx_item(const float *X, int64_t m, int64_t lda, int64_t ldx, int r,
                          const float *W, int rs, float *A, void *ws, unsigned int *tickets,
                          WtxItem *it, int64_t *ctas) {
    SplitPlan sp{};
    cudaError_t e = cudaErrorInvalidValue;
    switch (rs) {
#define NMF_WTX_PLAN(RV)                            \
    case RV:                                        \
        e = wtx_prepare<RV>(&sp, m, lda);           \
        break;
        NMF_WTX_PLAN(8) NMF_WTX_PLAN(16) NMF_WTX_PLAN(24) NMF_WTX_PLAN(32)
        NMF_WTX_PLAN(40) NMF_WTX_PLAN(48) NMF_WTX_PLAN(56) NMF_WTX_PLAN(64)
        NMF_WTX_PLAN(72) NMF_WTX_PLAN(80) NMF_WTX_PLAN(88) NMF_WTX_PLAN(96)
        NMF_WTX_PLAN(104) NMF_WTX_PLAN(112) NMF_WTX_PLAN(120) NMF_WTX_PLAN(128)
#undef NMF_WTX_PLAN
        default: break;
    }
    if (e != cudaSuccess) return e;
    *it = WtxItem{X, m, ldx, r, W, A, lda, sp.per_split, static_cast<float *>(ws), tickets,
                  sp.tiles, sp.nsplit};
    *ctas = sp.tiles * sp.nsplit;
    return cudaSuccess;
}

cudaError_t launch_wtx_grouped(int key, const WtxItem *items, const int64_t *begin, int nitems,
                               int64_t ctas, cudaStream_t st) {
    if (nitems < 1 || ctas < 1) return cudaSuccess;
    switch (key) {
#define NMF_WTX_GROUPED(RV)                                                                  \
    case RV:                                                                                 \
        wtx_f32_grouped<RV><<<(unsigned)ctas, 4 * RV, wtx_smem<RV>(), st>>>(items, begin,     \
                                                                           nitems);           \
        return cudaGetLastError();
        NMF_WTX_GROUPED(8) NMF_WTX_GROUPED(16) NMF_WTX_GROUPED(24) NMF_WTX_GROUPED(32)
        NMF_WTX_GROUPED(40) NMF_WTX_GROUPED(48) NMF_WTX_GROUPED(56) NMF_WTX_GROUPED(64)
        NMF_WTX_GROUPED(72) NMF_WTX_GROUPED(80) NMF_WTX_GROUPED(88) NMF_WTX_GROUPED(96)
        NMF_WTX_GROUPED(104) NMF_WTX_GROUPED(112) NMF_WTX_GROUPED(120) NMF_WTX_GROUPED(128)
#undef NMF_WTX_GROUPED
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t plan_xht_item(const float *X, int64_t m, int64_t ldx, int r, const float *H,
                          int64_t ldh, float *C, float *C_lo, int rs, void *ws,
                          unsigned int *tickets, XhtItem *it, int64_t *ctas) {
    const bool big = xht_big(m, r);
    SplitPlan sp{};
    cudaError_t e = cudaErrorInvalidValue;
    switch ((r + 7) / 8) {
#define NMF_XHT_PLAN(TRV)                                                                    \
    case TRV:                                                                                \
        e = big ? xht_prepare<4, TRV>(&sp, m, ldx) : xht_prepare<2, TRV>(&sp, m, ldx);       \
        break;
        NMF_XHT_PLAN(1) NMF_XHT_PLAN(2) NMF_XHT_PLAN(3) NMF_XHT_PLAN(4)
        NMF_XHT_PLAN(5) NMF_XHT_PLAN(6) NMF_XHT_PLAN(7) NMF_XHT_PLAN(8)
        NMF_XHT_PLAN(9) NMF_XHT_PLAN(10) NMF_XHT_PLAN(11) NMF_XHT_PLAN(12)
        NMF_XHT_PLAN(13) NMF_XHT_PLAN(14) NMF_XHT_PLAN(15) NMF_XHT_PLAN(16)
#undef NMF_XHT_PLAN
        default: break;
    }
    if (e != cudaSuccess) return e;
    *it = XhtItem{X, m, ldx, r, H, ldh, C, C_lo, rs, sp.per_split, static_cast<float *>(ws),
                  tickets, sp.tiles, sp.nsplit};
    *ctas = sp.tiles * sp.nsplit;
    return cudaSuccess;
}

cudaError_t launch_xht_grouped(int key, const XhtItem *items, const int64_t *begin, int nitems,
                               int64_t ctas, cudaStream_t st) {
    if (nitems < 1 || ctas < 1) return cudaSuccess;
    const int tm = key / 32, tr = key % 32;
    switch (tr) {
#define NMF_XHT_GROUPED(TRV)                                                                 \
    case TRV:                                                                                \
        if (tm == 4)                                                                         \
            xht_f32_grouped<4, TRV><<<(unsigned)ctas, kThreads, xht_smem<4, TRV>(), st>>>(    \
                items, begin, nitems);                                                       \
        else                                                                                 \
            xht_f32_grouped<2, TRV><<<(unsigned)ctas, kThreads, xht_smem<2, TRV>(), st>>>(    \
                items, begin, nitems);                                                       \
        return cudaGetLastError();
        NMF_XHT_GROUPED(1) NMF_XHT_GROUPED(2) NMF_XHT_GROUPED(3) NMF_XHT_GROUPED(4)
        NMF_XHT_GROUPED(5) NMF_XHT_GROUPED(6) NMF_XHT_GROUPED(7) NMF_XHT_GROUPED(8)
        NMF_XHT_GROUPED(9) NMF_XHT_GROUPED(10) NMF_XHT_GROUPED(11) NMF_XHT_GROUPED(12)
        NMF_XHT_GROUPED(13) NMF_XHT_GROUPED(14) NMF_XHT_GROUPED(15) NMF_XHT_GROUPED(16)
#undef NMF_XHT_GROUPED
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace nmfg
