// csr.cu -- the two X products for a sparse X (document matrices, Table 2 of
// Ang & Gillis, arXiv 1805.06604), without atomics:
//   C = X H_y^T : one warp per row of X (CSR); each nonzero X(i,j) gathers the
//                 contiguous row j of H_y^T (n x rs, built by transpose_h).
//   A = W_y^T X : one warp per column of X (CSC = CSR of X^T); each nonzero
//                 X(i,j) gathers the contiguous row i of W_y (m x rs).
// Lanes cover the rank dimension (lane, lane+32, ...), so every gather is a
// coalesced read of one factor row.  Sums run over the stored entries in
// index order, so results are deterministic.
#include <cuda_runtime.h>

#include "common.cuh"

namespace nmfg {
namespace {

constexpr int kWarps = 8;

template <int E>
__global__ void __launch_bounds__(kWarps * 32)
spmm_rows_kernel(const int64_t *__restrict__ ptr, const int32_t *__restrict__ idx,
                 const float *__restrict__ val, int64_t rows, int r, int rs,
                 const float *__restrict__ F,           // gathered factor, (cols) x rs
                 float *__restrict__ out, int64_t out_row_stride, int64_t out_col_stride) {
    const int lane = threadIdx.x % 32;
    const int64_t row = (int64_t)blockIdx.x * kWarps + threadIdx.x / 32;
    if (row >= rows) return;
    float acc[E];
#pragma unroll
    for (int e = 0; e < E; ++e) acc[e] = 0.0f;
    const int64_t p0 = ptr[row], p1 = ptr[row + 1];
    for (int64_t base = p0; base < p1; base += 32) {
        const int64_t q = base + lane;
        const int32_t c = q < p1 ? idx[q] : 0;
        const float v = q < p1 ? val[q] : 0.0f;
        const int cnt = (p1 - base) < 32 ? (int)(p1 - base) : 32;
        for (int u = 0; u < cnt; ++u) {
            const int32_t cu = __shfl_sync(0xffffffffu, c, u);
            const float vu = __shfl_sync(0xffffffffu, v, u);
            const float *f = F + (int64_t)cu * rs;
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int k = lane + 32 * e;
                if (k < rs) acc[e] = fmaf(vu, f[k], acc[e]);
            }
        }
    }
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int k = lane + 32 * e;
        if (k < r) out[row * out_row_stride + (int64_t)k * out_col_stride] = acc[e];
        else if (k < rs && out_col_stride == 1) out[row * out_row_stride + k] = 0.0f;
    }
}

template <int E>
cudaError_t spmm_launch(const int64_t *ptr, const int32_t *idx, const float *val, int64_t rows,
                        int r, int rs, const float *F, float *out, int64_t ors, int64_t ocs,
                        cudaStream_t st) {
    const unsigned grid = (unsigned)((rows + kWarps - 1) / kWarps);
    if (grid == 0) return cudaSuccess;
    spmm_rows_kernel<E><<<grid, kWarps * 32, 0, st>>>(ptr, idx, val, rows, r, rs, F, out, ors, ocs);
    return cudaGetLastError();
}

cudaError_t spmm(const int64_t *ptr, const int32_t *idx, const float *val, int64_t rows, int r,
                 int rs, const float *F, float *out, int64_t ors, int64_t ocs, cudaStream_t st) {
    switch ((rs + 31) / 32) {
        case 1: return spmm_launch<1>(ptr, idx, val, rows, r, rs, F, out, ors, ocs, st);
        case 2: return spmm_launch<2>(ptr, idx, val, rows, r, rs, F, out, ors, ocs, st);
        case 3: return spmm_launch<3>(ptr, idx, val, rows, r, rs, F, out, ors, ocs, st);
        case 4: return spmm_launch<4>(ptr, idx, val, rows, r, rs, F, out, ors, ocs, st);
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

cudaError_t launch_xht_csr(const int64_t *rowptr, const int32_t *colidx, const float *val,
                           int64_t m, int r, int rs, const float *Ht, float *C, cudaStream_t st) {
    return spmm(rowptr, colidx, val, m, r, rs, Ht, C, rs, 1, st);
}

cudaError_t launch_wtx_csc(const int64_t *colptr, const int32_t *rowidx, const float *val,
                           int64_t n, int r, int rs, const float *W, float *A, int64_t lda,
                           cudaStream_t st) {
    return spmm(colptr, rowidx, val, n, r, rs, W, A, 1, lda, st);
}

cudaError_t launch_transpose_h(const float *H, int r, int64_t n, int64_t ldh, float *Ht, int rs,
                               cudaStream_t st) {
    dim3 grid((unsigned)((n + 31) / 32), (unsigned)((rs + 31) / 32));
    transpose_h_kernel<<<grid, dim3(32, 8), 0, st>>>(H, r, n, ldh, Ht, rs);
    return cudaGetLastError();
}

}  // namespace nmfg
