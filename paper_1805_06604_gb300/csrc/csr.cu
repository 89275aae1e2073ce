// csr.cu -- the two X products for a sparse X (document matrices, Table 2 of
// Ang & Gillis, arXiv 1805.06604), without atomics and deterministic:
//   C = X H_y^T : rows of X (CSR); each nonzero X(i,j) gathers the
//                 contiguous row j of H_y^T (n x rs, built by transpose_h);
//   A = W_y^T X : rows of X^T (the CSC copy); each nonzero X(i,j) gathers
//                 the contiguous row i of W_y (m x rs).
// Work is split by nonzeros, not by rows: warp c owns the stored entries
// [c*kChunk, (c+1)*kChunk), so the Zipf-heavy rows of a term-document
// matrix spread over many warps.  Lanes cover the rank dimension (lane,
// lane+32, ...), so every gather is one coalesced read of a factor row.
// A row that lies entirely inside a chunk is written directly.  A row cut
// by chunk boundaries leaves one partial per chunk it touches -- the tail of
// the chunk it starts in, and the head of every later chunk -- and a fix-up
// pass adds them in chunk order.  Rows without entries are zeroed first.
#include <cuda_runtime.h>

#include "common.cuh"

namespace nmfg {
namespace {

constexpr int kWarps = 8;
constexpr int64_t kChunk = 256;

template <int E>
__device__ __forceinline__ void store_vec(float *dst, int64_t col_stride, const float (&acc)[E],
                                          int lane, int r) {
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int k = lane + 32 * e;
        if (k < r) dst[(int64_t)k * col_stride] = acc[e];
    }
}

// out[row * ors + k * ocs] = sum_{q in row} val[q] * F[idx[q] * rs + k].
// seg[q] is the row of stored entry q (expanded from ptr at creation), so a
// row change is a register comparison, not a dependent load of ptr.
// head[c] / tail[c] (rs floats each) receive the partials of rows cut by the
// chunk boundaries.
template <int E>
__global__ void __launch_bounds__(kWarps * 32)
spmm_chunks_kernel(const int64_t *__restrict__ ptr, const int32_t *__restrict__ idx,
                   const int32_t *__restrict__ seg, const float *__restrict__ val, int64_t nnz,
                   int r, int rs, const float *__restrict__ F, float *__restrict__ out,
                   int64_t ors, int64_t ocs, float *__restrict__ head, float *__restrict__ tail) {
    const int lane = threadIdx.x % 32;
    const int64_t c = (int64_t)blockIdx.x * kWarps + threadIdx.x / 32;
    const int64_t q0 = c * kChunk;
    if (q0 >= nnz) return;
    const int n_here = (int)(nnz - q0 < kChunk ? nnz - q0 : kChunk);
    int64_t row = seg[q0];
    bool started_before = ptr[row] < q0;
    float acc[E];
#pragma unroll
    for (int e = 0; e < E; ++e) acc[e] = 0.0f;
    bool kok[E];
#pragma unroll
    for (int e = 0; e < E; ++e) kok[e] = lane + 32 * e < rs;

    auto flush = [&](bool continues) {
        float *dst;
        int64_t stride = 1;
        if (started_before) {
            dst = head + c * rs;
        } else if (continues) {
            dst = tail + c * rs;
        } else {
            dst = out + row * ors;
            stride = ocs;
        }
        store_vec<E>(dst, stride, acc, lane, r);
#pragma unroll
        for (int e = 0; e < E; ++e) acc[e] = 0.0f;
    };

    // The factor rows of kBatch entries are gathered before any of them is
    // used, so their L2 latencies overlap instead of adding up.
    constexpr int kBatch = E <= 2 ? 8 : 4;
    for (int base = 0; base < n_here; base += 32) {
        const int ql = base + lane;
        const bool in = ql < n_here;
        const int32_t cidx = in ? idx[q0 + ql] : 0;
        const float v = in ? val[q0 + ql] : 0.0f;
        const int32_t rw = in ? seg[q0 + ql] : -1;
        const int cnt = n_here - base < 32 ? n_here - base : 32;
        for (int u0 = 0; u0 < cnt; u0 += kBatch) {
            float fv[kBatch][E];
#pragma unroll
            for (int j = 0; j < kBatch; ++j) {
                const int32_t cu = __shfl_sync(0xffffffffu, cidx, (u0 + j) & 31);
                const float *f = F + (int64_t)cu * rs;
#pragma unroll
                for (int e = 0; e < E; ++e) fv[j][e] = kok[e] ? __ldg(f + lane + 32 * e) : 0.0f;
            }
#pragma unroll
            for (int j = 0; j < kBatch; ++j) {
                const float vu = __shfl_sync(0xffffffffu, v, (u0 + j) & 31);
                const int32_t ru = __shfl_sync(0xffffffffu, rw, (u0 + j) & 31);
                if (u0 + j < cnt) {
                    if (ru != row) {                         // the previous row ends here
                        flush(false);
                        started_before = false;
                        row = ru;
                    }
#pragma unroll
                    for (int e = 0; e < E; ++e)
                        if (kok[e]) acc[e] = fmaf(vu, fv[j][e], acc[e]);
                }
            }
        }
    }
    flush(ptr[row + 1] > q0 + n_here);
}

// For every chunk whose last row starts inside it and continues past it:
// tail[c] + head[c+1] + ... + head[c_end] in chunk order.
template <int E>
__global__ void __launch_bounds__(kWarps * 32)
spmm_fixup_kernel(const int64_t *__restrict__ ptr, const int32_t *__restrict__ seg, int64_t nnz,
                  int r, int rs, float *__restrict__ out, int64_t ors, int64_t ocs,
                  const float *__restrict__ head, const float *__restrict__ tail) {
    const int lane = threadIdx.x % 32;
    const int64_t c = (int64_t)blockIdx.x * kWarps + threadIdx.x / 32;
    const int64_t q0 = c * kChunk;
    if (q0 >= nnz) return;
    const int64_t q1 = min(nnz, q0 + kChunk);
    const int64_t row = seg[q1 - 1];
    if (ptr[row + 1] <= q1 || ptr[row] < q0) return;   // not a row that starts here and continues
    const int64_t c_end = (ptr[row + 1] - 1) / kChunk;
    float acc[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int k = lane + 32 * e;
        acc[e] = k < rs ? tail[c * rs + k] : 0.0f;
    }
    // In chunk order; the loads of eight chunks go out together (a row of
    // a frequent term spans many chunks).
#pragma unroll 8
    for (int64_t cc = c + 1; cc <= c_end; ++cc) {
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int k = lane + 32 * e;
            if (k < rs) acc[e] += head[cc * rs + k];
        }
    }
    store_vec<E>(out + row * ors, ocs, acc, lane, r);
}

template <int E>
cudaError_t spmm_launch(const int64_t *ptr, const int32_t *idx, const int32_t *seg,
                        const float *val, int64_t rows, int64_t nnz, int r, int rs, const float *F,
                        float *out, int64_t ors, int64_t ocs, float *head, float *tail,
                        cudaStream_t st) {
    (void)rows;
    const int64_t chunks = (nnz + kChunk - 1) / kChunk;
    const unsigned grid = (unsigned)((chunks + kWarps - 1) / kWarps);
    if (grid == 0) return cudaSuccess;
    spmm_chunks_kernel<E><<<grid, kWarps * 32, 0, st>>>(ptr, idx, seg, val, nnz, r, rs, F, out,
                                                        ors, ocs, head, tail);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    spmm_fixup_kernel<E><<<grid, kWarps * 32, 0, st>>>(ptr, seg, nnz, r, rs, out, ors, ocs, head,
                                                       tail);
    return cudaGetLastError();
}

cudaError_t spmm(const int64_t *ptr, const int32_t *idx, const int32_t *seg, const float *val,
                 int64_t rows, int64_t nnz, int r, int rs, const float *F, float *out, int64_t ors,
                 int64_t ocs, float *head, float *tail, cudaStream_t st) {
    switch ((rs + 31) / 32) {
#define NMF_SPMM_CASE(EV)                                                                     \
    case EV:                                                                                  \
        return spmm_launch<EV>(ptr, idx, seg, val, rows, nnz, r, rs, F, out, ors, ocs, head,   \
                               tail, st);
        NMF_SPMM_CASE(1) NMF_SPMM_CASE(2) NMF_SPMM_CASE(3) NMF_SPMM_CASE(4)
#undef NMF_SPMM_CASE
        default: return cudaErrorInvalidValue;
    }
}

// Ht[j * rs + k] = H[k * ldh + j]; 32 x 32 tiles through shared memory.
__global__ void transpose_h_kernel(const float *__restrict__ H, int r, int64_t n, int64_t ldh,
                                   float *__restrict__ Ht, int rs) {
    __shared__ float tile[32][33];
    const int64_t j0 = (int64_t)blockIdx.x * 32;
    const int k0 = blockIdx.y * 32;
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
        const int k = k0 + y;
        const int64_t j = j0 + threadIdx.x;
        tile[y][threadIdx.x] = (k < r && j < n) ? H[(int64_t)k * ldh + j] : 0.0f;
    }
    __syncthreads();
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
        const int64_t j = j0 + y;
        const int k = k0 + threadIdx.x;
        if (j < n && k < rs) Ht[j * rs + k] = tile[threadIdx.x][y];
    }
}

}  // namespace

size_t csr_carry_floats(int64_t nnz, int rs) {
    const int64_t chunks = (nnz + kChunk - 1) / kChunk;
    return (size_t)(chunks > 0 ? chunks : 1) * rs * 2;
}

// C (m x rs) = X H^T; the whole of C is rewritten (rows without entries are 0).
cudaError_t launch_xht_csr(const int64_t *rowptr, const int32_t *colidx, const int32_t *rowseg,
                           const float *val, int64_t m, int64_t nnz, int r, int rs,
                           const float *Ht, float *C, float *carry, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(C, 0, sizeof(float) * (size_t)m * rs, st);
    if (e != cudaSuccess) return e;
    const size_t half = csr_carry_floats(nnz, rs) / 2;
    return spmm(rowptr, colidx, rowseg, val, m, nnz, r, rs, Ht, C, rs, 1, carry, carry + half,
                st);
}

// A (r x lda) = W^T X from the CSC copy; columns without entries are 0.
cudaError_t launch_wtx_csc(const int64_t *colptr, const int32_t *rowidx, const int32_t *colseg,
                           const float *val, int64_t n, int64_t nnz, int r, int rs,
                           const float *W, float *A, int64_t lda, float *carry, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(A, 0, sizeof(float) * (size_t)r * lda, st);
    if (e != cudaSuccess) return e;
    const size_t half = csr_carry_floats(nnz, rs) / 2;
    return spmm(colptr, rowidx, colseg, val, n, nnz, r, rs, W, A, 1, lda, carry, carry + half,
                st);
}

cudaError_t launch_transpose_h(const float *H, int r, int64_t n, int64_t ldh, float *Ht, int rs,
                               cudaStream_t st) {
    dim3 grid((unsigned)((n + 31) / 32), (unsigned)((rs + 31) / 32));
    transpose_h_kernel<<<grid, dim3(32, 8), 0, st>>>(H, r, n, ldh, Ht, rs);
    return cudaGetLastError();
}

}  // namespace nmfg
