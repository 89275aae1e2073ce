// tc_products.cu -- the X products on the 5th-generation tensor cores
// (precision modes NMF_PREC_TF32 and NMF_PREC_BF16X3).
//
// out = P Q^T with P (M x K) and Q (N x K) both K-major (rows contiguous in
// K), N <= 128.  Used as C = X H_y^T (P = X, Q = H_y) and as A^T = X^T W_y
// (P = X^T, a transposed copy of X kept for these modes, Q = W_y^T).
//
// Per CTA: one 128-row tile of P, all N columns, a range of K (split-K).
// Tiles arrive by TMA (cp.async.bulk.tensor, 128-byte swizzle) into a
// 4-stage shared-memory ring; one thread issues tcgen05.mma into an FP32
// accumulator in tensor memory; after the last K step the four warps read
// their 32 TMEM lanes (tcgen05.ld) and write the tile.  Split partials are
// summed in split order by the last CTA of a row tile (atomic ticket).
//
//  TF32:     D += P Q^T with the operands read as TF32 (one product).
//  BF16X3:   P and Q are held as hi/lo BF16 pairs (x ~ hi + lo); three
//            products hi.hi + hi.lo + lo.hi accumulate in FP32.
//
// Every mbarrier wait is bounded; a wait that runs out sets *err_flag, the
// CTA skips the rest of its work, frees its tensor memory and returns.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include "common.cuh"

namespace nmfg {
namespace {

constexpr int kThreads = 128;
constexpr int kBM = 128;
constexpr int kAtom = 128;                      // bytes per swizzled row
constexpr unsigned long long kSpinLimit = 1ull << 26;

// ------------------------------------------------------------ PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

// Bounded wait for phase `parity`; false (and *err = 1) when it runs out.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, int *err) {
    const uint32_t a = smem_u32(bar);
    for (unsigned long long i = 0; i < kSpinLimit; ++i) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    atomicExch(err, 1);
    return false;
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int c0, int c1,
                                            uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
        "l"((unsigned long long)map), "r"(c0), "r"(c1), "r"(smem_u32(bar))
        : "memory");
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, rows of 128
// bytes, 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFF) >> 4);          // start address
    d |= (uint64_t)1 << 16;                          // leading byte offset (unused here)
    d |= (uint64_t)(1024 >> 4) << 32;                // stride byte offset
    d |= (uint64_t)1 << 46;                          // descriptor version
    d |= (uint64_t)2 << 61;                          // 128-byte swizzle
    return d;
}

// Instruction descriptor: FP32 accumulate, K-major A and B, M x N.
__host__ __device__ constexpr uint32_t instr_desc(int ab_format, int M, int N) {
    return (1u << 4) | ((uint32_t)ab_format << 7) | ((uint32_t)ab_format << 10) |
           ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

template <int KIND>
__device__ __forceinline__ void mma(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t idesc,
                                    uint32_t accumulate) {
    if constexpr (KIND == 0) {
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
            "l"(da), "l"(db), "r"(idesc), "r"(accumulate));
    } else {
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
            "l"(da), "l"(db), "r"(idesc), "r"(accumulate));
    }
}

__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(bar))
        : "memory");
}

// 32 lanes x 32 bits, 16 consecutive columns.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

template <int KIND, int N>
struct TcCfg {
    static constexpr int kElem = KIND == 0 ? 4 : 2;            // bytes per element
    static constexpr int kBK = kAtom / kElem;                  // K elements per stage
    static constexpr int kPBytes = kBM * kAtom;                // one P tile
    static constexpr int kQBytes = N * kAtom;                  // one Q tile
    static constexpr int kParts = KIND == 0 ? 1 : 2;           // hi (and lo)
    static constexpr int kStageBytes = kParts * (kPBytes + kQBytes);
    static constexpr int kKSteps = kAtom / 32;                 // MMAs of 32 bytes of K
    static constexpr uint32_t kIdesc = instr_desc(KIND == 0 ? 2 : 1, kBM, N);
    static constexpr int kTmemCols = N <= 32 ? 32 : (N <= 64 ? 64 : 128);
    static constexpr int kStages = (4 * kStageBytes <= 200 * 1024) ? 4 : (200 * 1024) / kStageBytes;
};

template <int KIND, int N, bool TRANS_OUT>
__global__ void __launch_bounds__(kThreads, 1)
tc_gemm_kernel(const __grid_constant__ CUtensorMap map_p, const __grid_constant__ CUtensorMap map_q,
               const __grid_constant__ CUtensorMap map_p_lo,
               const __grid_constant__ CUtensorMap map_q_lo, int64_t M, int64_t K, int nvalid,
               float *__restrict__ out, int64_t out_ld, int64_t k_per_split,
               float *__restrict__ part, unsigned int *__restrict__ tickets, int *err_flag) {
    using Cfg = TcCfg<KIND, N>;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *smem = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    constexpr int kStages = Cfg::kStages;
    __shared__ __align__(8) uint64_t full_bar[kStages], empty_bar[kStages], done_bar;
    __shared__ uint32_t tmem_base_sh;
    __shared__ int skip_sh;
    __shared__ bool am_last;

    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int64_t row0 = (int64_t)blockIdx.x * kBM;
    const int split = blockIdx.y, nsplit = gridDim.y;
    const int64_t kbeg = (int64_t)split * k_per_split;
    const int64_t kend = min(K, kbeg + k_per_split);
    const int nk = kend > kbeg ? (int)((kend - kbeg + Cfg::kBK - 1) / Cfg::kBK) : 0;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full_bar[s], 1);
            mbar_init(&empty_bar[s], 1);
        }
        mbar_init(&done_bar, 1);
        skip_sh = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_base_sh)),
                     "r"(Cfg::kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base_sh;

    if (threadIdx.x == 0 && nk > 0) {
        // TMA producer.
        for (int it = 0; it < nk; ++it) {
            const int s = it % kStages;
            if (it >= kStages && !mbar_wait(&empty_bar[s], ((it / kStages) - 1) & 1, err_flag)) {
                skip_sh = 1;
                break;
            }
            unsigned char *st = smem + s * Cfg::kStageBytes;
            const int k0 = (int)(kbeg + (int64_t)it * Cfg::kBK);
            mbar_expect_tx(&full_bar[s], Cfg::kStageBytes);
            tma_load_2d(st, &map_p, k0, (int)row0, &full_bar[s]);
            tma_load_2d(st + Cfg::kPBytes, &map_q, k0, 0, &full_bar[s]);
            if constexpr (KIND == 1) {
                tma_load_2d(st + Cfg::kPBytes + Cfg::kQBytes, &map_p_lo, k0, (int)row0,
                            &full_bar[s]);
                tma_load_2d(st + 2 * Cfg::kPBytes + Cfg::kQBytes, &map_q_lo, k0, 0,
                            &full_bar[s]);
            }
        }
    } else if (threadIdx.x == 32 && nk > 0) {
        // MMA issuer.
        for (int it = 0; it < nk; ++it) {
            const int s = it % kStages;
            if (!mbar_wait(&full_bar[s], (it / kStages) & 1, err_flag)) {
                skip_sh = 1;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t base = smem_u32(smem + s * Cfg::kStageBytes);
            const uint32_t p_hi = base, q_hi = base + Cfg::kPBytes;
#pragma unroll
            for (int ks = 0; ks < Cfg::kKSteps; ++ks) {
                const uint32_t off = ks * 32;
                const uint32_t acc = (it > 0 || ks > 0) ? 1u : 0u;
                mma<KIND>(tmem, smem_desc(p_hi + off), smem_desc(q_hi + off), Cfg::kIdesc, acc);
                if constexpr (KIND == 1) {
                    const uint32_t p_lo = base + Cfg::kPBytes + Cfg::kQBytes;
                    const uint32_t q_lo = p_lo + Cfg::kPBytes;
                    mma<KIND>(tmem, smem_desc(p_hi + off), smem_desc(q_lo + off), Cfg::kIdesc, 1u);
                    mma<KIND>(tmem, smem_desc(p_lo + off), smem_desc(q_hi + off), Cfg::kIdesc, 1u);
                }
            }
            mma_commit(&empty_bar[s]);
        }
        mma_commit(&done_bar);
    }
    __syncthreads();

    // Epilogue: warp w owns TMEM lanes (rows) 32w .. 32w+31.
    float *my_part = nullptr;
    const bool have_result = nk > 0 && !skip_sh && mbar_wait(&done_bar, 0, err_flag);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const int64_t row = row0 + warp * 32 + lane;
    if (nsplit > 1) my_part = part + ((int64_t)blockIdx.x * nsplit + split) * (kBM * N);
#pragma unroll
    for (int c0 = 0; c0 < N; c0 += 16) {
        float v[16];
        if (have_result) {
            tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
        } else {
#pragma unroll
            for (int i = 0; i < 16; ++i) v[i] = 0.0f;
        }
        if (nsplit > 1) {
            float *dst = my_part + (int64_t)(warp * 32 + lane) * N + c0;
#pragma unroll
            for (int i = 0; i < 16; i += 4)
                *reinterpret_cast<float4 *>(dst + i) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
        } else if (row < M) {
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const int col = c0 + i;
                if (col < nvalid) {
                    if (TRANS_OUT) out[(int64_t)col * out_ld + row] = v[i];
                    else out[row * out_ld + col] = v[i];
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(Cfg::kTmemCols)
                     : "memory");
    if (nsplit == 1) return;

    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned int t = atomicAdd(tickets + blockIdx.x, 1u);
        am_last = (t == (unsigned)nsplit - 1);
    }
    __syncthreads();
    if (!am_last) return;
    __threadfence();
    const float *base = part + (int64_t)blockIdx.x * nsplit * (kBM * N);
    for (int e = threadIdx.x; e < kBM * N; e += kThreads) {
        float s = 0.0f;
        for (int q = 0; q < nsplit; ++q) s += __ldcg(base + (int64_t)q * kBM * N + e);
        const int64_t r_ = row0 + e / N;
        const int col = e % N;
        if (r_ < M && col < nvalid) {
            if (TRANS_OUT) out[(int64_t)col * out_ld + r_] = s;
            else out[r_ * out_ld + col] = s;
        }
    }
    if (threadIdx.x == 0) tickets[blockIdx.x] = 0u;
}

// ------------------------------------------------------------ host side
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// 2-D map of a rows x cols matrix (row stride ld elements), box box_rows x
// (128 bytes of columns), 128-byte swizzle, zero fill outside.
bool make_map(CUtensorMap *map, const void *ptr, bool bf16, int64_t rows, int64_t cols, int64_t ld,
              int box_rows) {
    auto fn = encode_fn();
    if (!fn) return false;
    const int esz = bf16 ? 2 : 4;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)(ld * esz)};
    cuuint32_t box[2] = {(cuuint32_t)(kAtom / esz), (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(map, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                    2, const_cast<void *>(ptr), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

struct TcPlan {
    int nsplit;
    int64_t tiles, k_per_split;
};

TcPlan plan_tc(int64_t M, int64_t K, int bk) {
    TcPlan p;
    p.tiles = (M + kBM - 1) / kBM;
    int64_t want = (kNumSMs + p.tiles - 1) / p.tiles;               // ~1 CTA per SM
    const int64_t max_split = (K + 8 * bk - 1) / (8 * bk);
    if (want > max_split) want = max_split;
    if (want < 1) want = 1;
    if (want > 16) want = 16;
    p.k_per_split = ((K + want - 1) / want + bk - 1) / bk * bk;
    p.nsplit = (int)((K + p.k_per_split - 1) / p.k_per_split);
    return p;
}

template <int KIND, int N, bool TRANS>
cudaError_t tc_launch(const TcOperands &o, float *out, int64_t out_ld, void *ws,
                      unsigned int *tickets, int *err_flag, cudaStream_t st) {
    using Cfg = TcCfg<KIND, N>;
    const TcPlan p = plan_tc(o.M, o.K, Cfg::kBK);
    CUtensorMap mp, mq, mpl, mql;
    const bool bf = KIND == 1;
    // Q has q_rows <= N real rows; the N-row box reads zeros beyond them.
    if (!make_map(&mp, o.P, bf, o.M, o.K, o.ldp, kBM) ||
        !make_map(&mq, o.Q, bf, o.q_rows, o.K, o.ldq, N))
        return cudaErrorInvalidValue;
    if (bf) {
        if (!make_map(&mpl, o.P_lo, bf, o.M, o.K, o.ldp, kBM) ||
            !make_map(&mql, o.Q_lo, bf, o.q_rows, o.K, o.ldq, N))
            return cudaErrorInvalidValue;
    } else {
        mpl = mp;
        mql = mq;
    }
    const size_t smem = (size_t)Cfg::kStages * Cfg::kStageBytes + 1024;
    auto kern = tc_gemm_kernel<KIND, N, TRANS>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)p.tiles, (unsigned)p.nsplit);
    kern<<<grid, kThreads, smem, st>>>(mp, mq, mpl, mql, o.M, o.K, o.nvalid, out, out_ld,
                                       p.k_per_split, static_cast<float *>(ws), tickets,
                                       err_flag);
    return cudaGetLastError();
}

template <int KIND, bool TRANS>
cudaError_t tc_dispatch_n(const TcOperands &o, float *out, int64_t out_ld, void *ws,
                          unsigned int *tickets, int *err_flag, cudaStream_t st) {
    switch (o.N) {
        case 16: return tc_launch<KIND, 16, TRANS>(o, out, out_ld, ws, tickets, err_flag, st);
        case 32: return tc_launch<KIND, 32, TRANS>(o, out, out_ld, ws, tickets, err_flag, st);
        case 48: return tc_launch<KIND, 48, TRANS>(o, out, out_ld, ws, tickets, err_flag, st);
        case 64: return tc_launch<KIND, 64, TRANS>(o, out, out_ld, ws, tickets, err_flag, st);
        case 80: return tc_launch<KIND, 80, TRANS>(o, out, out_ld, ws, tickets, err_flag, st);
        case 96: return tc_launch<KIND, 96, TRANS>(o, out, out_ld, ws, tickets, err_flag, st);
        case 112: return tc_launch<KIND, 112, TRANS>(o, out, out_ld, ws, tickets, err_flag, st);
        case 128: return tc_launch<KIND, 128, TRANS>(o, out, out_ld, ws, tickets, err_flag, st);
        default: return cudaErrorInvalidValue;
    }
}

// hi = bf16(x), lo = bf16(x - hi), element-wise over rows x cols (row stride ld).
__global__ void split_bf16_kernel(const float *__restrict__ x, int64_t rows, int64_t cols,
                                  int64_t ld, __nv_bfloat16 *__restrict__ hi,
                                  __nv_bfloat16 *__restrict__ lo, int64_t ld_out) {
    const int64_t total = rows * cols;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = q / cols, j = q % cols;
        const float v = x[i * ld + j];
        const __nv_bfloat16 h = __float2bfloat16_rn(v);
        hi[i * ld_out + j] = h;
        lo[i * ld_out + j] = __float2bfloat16_rn(v - __bfloat162float(h));
    }
}

// out (cols x rows, row stride ld_out) = in^T (in: rows x cols, row stride ld_in).
__global__ void transpose_kernel(const float *__restrict__ in, int64_t rows, int64_t cols,
                                 int64_t ld_in, float *__restrict__ out, int64_t ld_out) {
    __shared__ float tile[32][33];
    const int64_t c0 = (int64_t)blockIdx.x * 32, r0 = (int64_t)blockIdx.y * 32;
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
        const int64_t r = r0 + y, c = c0 + threadIdx.x;
        tile[y][threadIdx.x] = (r < rows && c < cols) ? in[r * ld_in + c] : 0.0f;
    }
    __syncthreads();
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
        const int64_t c = c0 + y, r = r0 + threadIdx.x;
        if (c < cols && r < rows) out[c * ld_out + r] = tile[threadIdx.x][y];
    }
}

}  // namespace

size_t tc_ws_bytes(int64_t M, int64_t K, int N, int precision) {
    const TcPlan p = plan_tc(M, K, precision == NMF_PREC_TF32 ? 32 : 64);
    if (p.nsplit == 1) return 256;
    return sizeof(float) * (size_t)p.tiles * p.nsplit * kBM * N;
}

int64_t tc_num_tickets(int64_t M) { return (M + kBM - 1) / kBM; }

bool tc_available() { return encode_fn() != nullptr; }

cudaError_t launch_tc_product(const TcOperands &o, int precision, bool transposed_out, float *out,
                              int64_t out_ld, void *ws, unsigned int *tickets, int *err_flag,
                              cudaStream_t st) {
    if (precision == NMF_PREC_TF32)
        return transposed_out ? tc_dispatch_n<0, true>(o, out, out_ld, ws, tickets, err_flag, st)
                              : tc_dispatch_n<0, false>(o, out, out_ld, ws, tickets, err_flag, st);
    if (precision == NMF_PREC_BF16X3)
        return transposed_out ? tc_dispatch_n<1, true>(o, out, out_ld, ws, tickets, err_flag, st)
                              : tc_dispatch_n<1, false>(o, out, out_ld, ws, tickets, err_flag, st);
    return cudaErrorInvalidValue;
}

cudaError_t launch_split_bf16(const float *x, int64_t rows, int64_t cols, int64_t ld,
                              __nv_bfloat16 *hi, __nv_bfloat16 *lo, int64_t ld_out,
                              cudaStream_t st) {
    int64_t blocks = (rows * cols + 255) / 256;
    if (blocks > 8 * kNumSMs) blocks = 8 * kNumSMs;
    if (blocks < 1) blocks = 1;
    split_bf16_kernel<<<(unsigned)blocks, 256, 0, st>>>(x, rows, cols, ld, hi, lo, ld_out);
    return cudaGetLastError();
}

cudaError_t launch_transpose(const float *in, int64_t rows, int64_t cols, int64_t ld_in,
                             float *out, int64_t ld_out, cudaStream_t st) {
    dim3 grid((unsigned)((cols + 31) / 32), (unsigned)((rows + 31) / 32));
    transpose_kernel<<<grid, dim3(32, 8), 0, st>>>(in, rows, cols, ld_in, out, ld_out);
    return cudaGetLastError();
}

}  // namespace nmfg
