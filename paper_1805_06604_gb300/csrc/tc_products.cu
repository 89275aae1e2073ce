// tc_products.cu -- the X products on the 5th-generation tensor cores
// (precision modes NMF_PREC_TF32 and NMF_PREC_BF16X3).
//
// out = P Q^T with P (M x K) and Q (N x K) both K-major (rows contiguous in
// K), N <= 128.  Used as C = X H_y^T (P = X, Q = H_y) and as A^T = X^T W_y
// (P = X^T, a transposed copy of X kept for these modes, Q = W_y^T).
//
// Persistent stream-K kernel: one CTA per SM, each owning an equal share of
// the (128-row tile of P, 64-element K stage) units, so every SM streams the
// same number of bytes of X.  A stage (two 128-byte-wide boxes of P and Q)
// arrives by TMA (cp.async.bulk.tensor, 128-byte swizzle) into a shared-
// memory ring; one thread issues tcgen05.mma into FP32 accumulators in
// tensor memory.  Up to N = 64 each K stage has its own accumulator (four in
// flight), which four epilogue warps read (tcgen05.ld) and add into a
// compensated register sum; wider tiles accumulate a whole segment in one of
// two accumulators.  The epilogue writes the tile, or a partial of it that
// the tile's last CTA (atomic ticket) adds to the other partials in CTA
// order -- deterministic.
//
//  TF32:     D += P Q^T with the operands rounded to the nearest TF32 value
//            (X when it is packed, the factor by prep_*_kernel).
//  BF16X3:   P and Q are held as hi/lo BF16 pairs (x ~ hi + lo); three
//            products hi.hi + hi.lo + lo.hi accumulate in FP32.
//
// Every mbarrier wait is bounded; a wait that runs out sets *err_flag, the
// CTA skips the rest of its work, waits (bounded) for its copies and MMAs in
// flight, frees its tensor memory and returns.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include "common.cuh"

namespace nmfg {
namespace {

constexpr int kBM = 128;
constexpr int kAtom = 128;                      // bytes per swizzled row
constexpr unsigned long long kSpinLimit = 1ull << 26;

// Failure-detection hook (nmf_debug_set_fixup_stall): extra partials the
// last CTA of a shared tile waits for in its final segment -- when none of
// its copies or MMAs is in flight -- so a test can make that bounded wait
// run out without faulting anything.  0 in normal use.
__device__ int g_fixup_stall = 0;

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

// Bounded wait for a long phase (a whole accumulation): polls with a short
// sleep so that the waiting thread takes no issue slots or barrier-unit
// bandwidth from the producer and the MMA issuer.
__device__ __forceinline__ bool mbar_wait_sleep(uint64_t *bar, uint32_t parity, int *err) {
    const uint32_t a = smem_u32(bar);
    for (unsigned long long i = 0; i < (kSpinLimit >> 2); ++i) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
        __nanosleep(128);
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

// Contiguous global -> shared copy (16-byte aligned, size a multiple of 16).
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes,
                                          uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_u32(dst)),
        "l"((unsigned long long)src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// The same with an L2 eviction policy: the packed X is read exactly once per
// product and is marked to leave L2 first, so that streaming it does not
// push out the factors and the partials that are read again.
__device__ __forceinline__ uint64_t evict_first_policy() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
__device__ __forceinline__ void bulk_load_stream(void *dst, const void *src, uint32_t bytes,
                                                 uint64_t *bar, uint64_t pol) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint "
        "[%0], [%1], %2, [%3], %4;" ::"r"(smem_u32(dst)),
        "l"((unsigned long long)src), "r"(bytes), "r"(smem_u32(bar)), "l"(pol)
        : "memory");
}

// Nearest TF32 value of x (ties away from zero).  The MMA reads an FP32
// operand's top 19 bits, i.e. it truncates: on nonnegative data that is a
// bias of about -2^-11 relative in every product, which the Remark 1 error
// (a difference of nearly equal terms) turns into an offset of order
// 1e-3 ||X||^2.  Operands are rounded to nearest before they reach it.
__device__ __forceinline__ float tf32_rna(float x) {
    uint32_t u;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"(x));
    return __uint_as_float(u);
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
    static constexpr int kAtomK = kAtom / kElem;               // K elements per 128-byte atom
    static constexpr int kAtoms = KIND == 0 ? 2 : 1;           // K atoms per stage
    static constexpr int kParts = KIND == 0 ? 1 : 2;           // hi (and lo)
    static constexpr int kBoxes = kAtoms * kParts;             // P boxes (and Q boxes) per stage
    static constexpr int kBK = kAtoms * kAtomK;                // K elements per stage
    static constexpr int kPBytes = kBM * kAtom;                // one P box
    static constexpr int kQBytes = N * kAtom;                  // one Q box
    static constexpr int kStageBytes = kBoxes * (kPBytes + kQBytes);
    static constexpr int kKSteps = kAtom / 32;                 // MMAs per atom (32 bytes of K)
    static constexpr uint32_t kIdesc = instr_desc(KIND == 0 ? 2 : 1, kBM, N);
    static constexpr int kAccCols = N <= 32 ? 32 : (N <= 64 ? 64 : 128);   // one accumulator
    // Up to N = 64 every K stage gets a fresh accumulator, which the
    // epilogue adds into a compensated (Kahan) register sum: the tensor
    // core's FP32 accumulation then spans only the 64 K of one stage, and
    // the result is accurate to a few units of FP32 rounding whatever K.
    // Wider tiles (2N sum registers would not fit) accumulate a whole
    // segment in tensor memory.
    static constexpr bool kComp = N <= 64;
    static constexpr int kGroup = 1;                           // K stages per drained accumulator
    static constexpr int kNumAcc = kComp ? 4 : 2;              // accumulators in flight
    static constexpr int kTmemCols = kNumAcc * kAccCols;
    static constexpr int kFit = (200 * 1024) / kStageBytes;
    static constexpr int kStages = kFit < 2 ? 2 : (kFit > 6 ? 6 : kFit);
    static_assert(kStages * kStageBytes + 2048 <= 227 * 1024, "stage ring exceeds shared memory");
};

constexpr int kTcThreads = 192;   // warps 0-3: epilogue, warp 4: TMA producer, warp 5: MMA issuer
constexpr int kMaxContrib = 64;   // CTAs that may share one row tile

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void epilogue_sync() {
    asm volatile("bar.sync 1, 128;" ::: "memory");
}

// Writes columns c0 .. c0+CW-1 of one output row (values v[0..CW)):
// transposed (column-major, coalesced across the warp's rows) or row-major,
// as float4 words when `vec` (row stride and valid width multiples of 4).
template <int CW, bool TRANS_OUT>
__device__ __forceinline__ void store_row(const float (&v)[CW], int c0, int N, float *out,
                                          int64_t out_ld, int64_t row, int64_t M, int nvalid,
                                          bool vec) {
    (void)N;
    if (row >= M) return;
    if (!TRANS_OUT && vec) {
#pragma unroll
        for (int i = 0; i < CW; i += 4)
            if (c0 + i < nvalid)
                *reinterpret_cast<float4 *>(out + row * out_ld + c0 + i) =
                    make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
        return;
    }
#pragma unroll
    for (int i = 0; i < CW; ++i) {
        const int col = c0 + i;
        if (col < nvalid) {
            if (TRANS_OUT) out[(int64_t)col * out_ld + row] = v[i];
            else out[row * out_ld + col] = v[i];
        }
    }
}

// Stream-K schedule over the (row tile, K stage) units, tile-major: CTA c
// owns units [total*c/G, total*(c+1)/G), so every CTA of a single wave gets
// the same amount of X.  A CTA's range splits into segments, one per row
// tile it touches.
struct StreamK {
    int64_t total, G;
    int nk;
    __device__ int64_t begin(int64_t c) const { return total * c / G; }
    __device__ int64_t cta_of(int64_t u) const { return ((u + 1) * G - 1) / total; }
};

// The segments of one CTA's unit range [u0, u1) (one per row tile touched),
// in processing order: the shorter of the two end segments first, then the
// other, then the whole tiles between them.  End segments share their tile
// with other CTAs, so their epilogues (a partial, or the fix-up) run while
// later segments still stream; the last segment processed is, where there
// is one, a whole tile (a plain store).  `orig` is the segment's index in
// unit order, which names its partial slot.
struct SegList {
    int64_t u0, u1, t0;
    int n, nk;
    __device__ SegList(int64_t a, int64_t b, int k) : u0(a), u1(b), nk(k) {
        t0 = a / k;
        n = b > a ? (int)((b - 1) / k - t0 + 1) : 0;
    }
    __device__ void get(int p, int64_t &tile, int &ks0, int &ks1, int &orig) const {
        if (n == 1) {
            orig = 0;
        } else {
            const int64_t len_first = nk - u0 % nk, len_last = (u1 - 1) % nk + 1;
            const bool first_short = len_first <= len_last;
            orig = p == 0 ? (first_short ? 0 : n - 1) : p == 1 ? (first_short ? n - 1 : 0) : p - 1;
        }
        tile = t0 + orig;
        ks0 = orig == 0 ? (int)(u0 % nk) : 0;
        ks1 = orig == n - 1 ? (int)((u1 - 1) % nk + 1) : nk;
    }
};

// out = P Q^T (see the top of the file).  Warp-specialised: warp 4 lane 0
// streams stages of P and Q boxes by TMA into a ring; warp 5 lane 0 issues
// tcgen05.mma into one of two TMEM accumulators (alternating per segment);
// warps 0-3 drain a finished accumulator (tcgen05.ld, 32 rows each) and
// write the tile, or a partial of it plus an ordered fix-up by the last of
// the tile's CTAs.
template <int KIND, int N, bool TRANS_OUT>
__global__ void __launch_bounds__(kTcThreads, 1)
tc_gemm_kernel(const unsigned char *__restrict__ pk, const unsigned char *__restrict__ pk_lo,
               const __grid_constant__ CUtensorMap map_q,
               const __grid_constant__ CUtensorMap map_q_lo, int64_t M, int64_t tiles, int nk,
               int nvalid, float *__restrict__ out, int64_t out_ld, float *__restrict__ part,
               int seg_max, unsigned int *__restrict__ tickets, int *err_flag) {
    using Cfg = TcCfg<KIND, N>;
    constexpr int kStages = Cfg::kStages;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *smem = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) uint64_t full_bar[kStages], empty_bar[kStages];
    constexpr int kNumAcc = Cfg::kNumAcc;
    __shared__ __align__(8) uint64_t acc_full[kNumAcc], acc_empty[kNumAcc], drain_bar, fix_bar;
    __shared__ uint32_t tmem_base_sh;
    __shared__ int abort_sh, seg_ok_sh;
    __shared__ bool am_last_sh;
    __shared__ int64_t contrib_sh[kMaxContrib];

    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const StreamK sk{tiles * nk, (int64_t)gridDim.x, nk};
    // Row-major output rows can be written as float4 words when aligned.
    const bool vec_out = !TRANS_OUT && out_ld % 4 == 0 && nvalid % 4 == 0 &&
                         ((uintptr_t)out & 15) == 0;
    const SegList segs(sk.begin(blockIdx.x), sk.begin(blockIdx.x + 1), nk);

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full_bar[s], 1);
            mbar_init(&empty_bar[s], 1);
        }
        for (int b = 0; b < kNumAcc; ++b) {
            mbar_init(&acc_full[b], 1);
            mbar_init(&acc_empty[b], 4);
        }
        mbar_init(&drain_bar, 1);
        mbar_init(&fix_bar, 1);
        abort_sh = 0;
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

    if (warp == 4) {
        if (lane == 0) {
            // TMA producer: every K stage of every segment, in order.  X is
            // constant, so the first ring fill of P goes out before
            // griddepcontrol.wait (the kernel may start while its
            // predecessor, which writes Q, still runs); the Q boxes of those
            // stages follow the wait.
            int it = 0;
            bool ok = true, waited = false;
            int k0_def[kStages];
            const uint64_t pol_x = evict_first_policy();
            auto issue_q = [&](int s, int k0) {
                unsigned char *qs = smem + s * Cfg::kStageBytes + Cfg::kBoxes * Cfg::kPBytes;
#pragma unroll
                for (int b = 0; b < Cfg::kBoxes; ++b) {
                    // TF32: box b is K atom b.  BF16X3: box b is part b (hi, lo).
                    const int kb = KIND == 0 ? k0 + b * Cfg::kAtomK : k0;
                    const CUtensorMap *mq = (KIND == 1 && b == 1) ? &map_q_lo : &map_q;
                    tma_load_2d(qs + b * Cfg::kQBytes, mq, kb, 0, &full_bar[s]);
                }
            };
            auto release_q = [&]() {
                asm volatile("griddepcontrol.wait;" ::: "memory");
                for (int j = 0; j < it && j < kStages; ++j) issue_q(j, k0_def[j]);
                waited = true;
            };
            for (int sp = 0; ok && sp < segs.n; ++sp) {
                int64_t tile;
                int ks0, ks1, orig;
                segs.get(sp, tile, ks0, ks1, orig);
                for (int ks = ks0; ks < ks1; ++ks, ++it) {
                    const int s = it % kStages;
                    if (it == kStages && !waited) release_q();
                    if (it >= kStages &&
                        !mbar_wait(&empty_bar[s], ((it / kStages) - 1) & 1, err_flag)) {
                        abort_sh = 1;
                        ok = false;
                        break;
                    }
                    unsigned char *st = smem + s * Cfg::kStageBytes;
                    const int k0 = ks * Cfg::kBK;
                    mbar_expect_tx(&full_bar[s], Cfg::kStageBytes);
#pragma unroll
                    for (int b = 0; b < Cfg::kBoxes; ++b) {
                        // P comes from its packed copy: block (tile, atom) is one
                        // contiguous, already swizzled 16 KiB image.
                        const int64_t atom = (int64_t)ks * Cfg::kAtoms + (KIND == 0 ? b : 0);
                        const unsigned char *src = ((KIND == 1 && b == 1) ? pk_lo : pk) +
                                                   (tile * ((int64_t)nk * Cfg::kAtoms) + atom) *
                                                       Cfg::kPBytes;
                        bulk_load_stream(st + b * Cfg::kPBytes, src, Cfg::kPBytes, &full_bar[s],
                                         pol_x);
                    }
                    if (waited) issue_q(s, k0);
                    else k0_def[s] = k0;
                }
            }
            if (!waited) release_q();
            // Copies still in flight (after an abort) land before the CTA exits.
            for (int j = it - kStages < 0 ? 0 : it - kStages; j < it; ++j)
                mbar_wait(&full_bar[j % kStages], (j / kStages) & 1, err_flag);
        }
    } else if (warp == 5) {
        if (lane == 0) {
            // MMA issuer.
            int it = 0, seg = 0, grp = 0;
            bool ok = true;
            for (; ok && seg < segs.n; ++seg) {
                int64_t tile;
                int ks0, ks1, orig;
                segs.get(seg, tile, ks0, ks1, orig);
                // Accumulator of the segment (kComp: of each stage, below).
                int b = seg % kNumAcc;
                if (!Cfg::kComp && seg >= kNumAcc &&
                    !mbar_wait(&acc_empty[b], ((seg / kNumAcc) - 1) & 1, err_flag)) {
                    abort_sh = 1;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                uint32_t d = tmem + (uint32_t)(b * Cfg::kAccCols);
                for (int ks = ks0; ks < ks1; ++ks, ++it) {
                    const int s = it % kStages;
                    // kComp: a group of kGroup stages (cut at the segment's
                    // end) accumulates into accumulator grp % kNumAcc.
                    const bool g_first = (ks - ks0) % Cfg::kGroup == 0;
                    const bool g_last = (ks - ks0) % Cfg::kGroup == Cfg::kGroup - 1 || ks == ks1 - 1;
                    if constexpr (Cfg::kComp) {
                        if (g_first) {
                            b = grp % kNumAcc;
                            d = tmem + (uint32_t)(b * Cfg::kAccCols);
                            if (grp >= kNumAcc &&
                                !mbar_wait(&acc_empty[b], ((grp / kNumAcc) - 1) & 1, err_flag)) {
                                abort_sh = 1;
                                ok = false;
                                break;
                            }
                        }
                    }
                    if (!mbar_wait(&full_bar[s], (it / kStages) & 1, err_flag)) {
                        abort_sh = 1;
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t base = smem_u32(smem + s * Cfg::kStageBytes);
                    const uint32_t qbase = base + Cfg::kBoxes * Cfg::kPBytes;
#pragma unroll
                    for (int a = 0; a < Cfg::kAtoms; ++a) {
#pragma unroll
                        for (int kk = 0; kk < Cfg::kKSteps; ++kk) {
                            const uint32_t off = kk * 32;
                            const uint32_t acc =
                                ((Cfg::kComp ? !g_first : ks > ks0) || a > 0 || kk > 0) ? 1u : 0u;
                            const uint32_t ph = base + a * Cfg::kPBytes + off;
                            const uint32_t qh = qbase + a * Cfg::kQBytes + off;
                            mma<KIND>(d, smem_desc(ph), smem_desc(qh), Cfg::kIdesc, acc);
                            if constexpr (KIND == 1) {
                                const uint32_t pl = base + Cfg::kPBytes + off;
                                const uint32_t ql = qbase + Cfg::kQBytes + off;
                                mma<KIND>(d, smem_desc(ph), smem_desc(ql), Cfg::kIdesc, 1u);
                                mma<KIND>(d, smem_desc(pl), smem_desc(qh), Cfg::kIdesc, 1u);
                            }
                        }
                    }
                    mma_commit(&empty_bar[s]);
                    if constexpr (Cfg::kComp) {
                        if (g_last) {
                            mma_commit(&acc_full[b]);
                            ++grp;
                        }
                    }
                }
                if (!ok) break;
                if constexpr (!Cfg::kComp) mma_commit(&acc_full[b]);
            }
            // Every MMA issued so far has completed before TMEM is freed.
            mma_commit(&drain_bar);
            mbar_wait(&drain_bar, 0, err_flag);
        }
    } else {
        // Epilogue warps 0-3: warp w owns TMEM lanes (tile rows) 32w .. 32w+31.
        int seg = 0, it = 0, grp = 0;
        bool fix_used = false;          // fix_bar serves one staged fix-up
        const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
        // One accumulator is complete (bounded wait by one thread, in warp 2:
        // a scheduler that neither the producer, warp 4, nor the MMA issuer,
        // warp 5, uses); the flag reaches all four warps.
        auto acc_ready = [&](int b, uint32_t parity, bool sleep) -> bool {
            if (threadIdx.x == 64)
                seg_ok_sh = sleep ? mbar_wait_sleep(&acc_full[b], parity, err_flag)
                                  : mbar_wait(&acc_full[b], parity, err_flag);
            epilogue_sync();
            const int ok = seg_ok_sh;
            epilogue_sync();            // all four warps read the flag before it is rewritten
            if (ok) asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            return ok != 0;
        };
        auto acc_release = [&](int b) {
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(&acc_empty[b]);
        };
        for (; seg < segs.n; ++seg) {
            int64_t tile;
            int ks0, ks1, orig;
            segs.get(seg, tile, ks0, ks1, orig);
            float v[N];
            bool seg_ok = true;
            if constexpr (Cfg::kComp) {
                // Each stage's accumulator is added into sum - cor (Kahan).
                float sum[N], cor[N];
#pragma unroll
                for (int i = 0; i < N; ++i) sum[i] = cor[i] = 0.0f;
                for (int ks = ks0; ks < ks1; ++ks, ++it) {
                    if (!((ks - ks0) % Cfg::kGroup == Cfg::kGroup - 1 || ks == ks1 - 1)) continue;
                    const int b = grp % kNumAcc;
                    const uint32_t par = (grp / kNumAcc) & 1;
                    ++grp;
                    if (!acc_ready(b, par, false)) {
                        seg_ok = false;
                        break;
                    }
#pragma unroll
                    for (int c0 = 0; c0 < N; c0 += 16) {
                        float w16[16];
                        tmem_ld16(lane_base + (uint32_t)(b * Cfg::kAccCols + c0), w16);
#pragma unroll
                        for (int i = 0; i < 16; ++i) {
                            const float y = w16[i] - cor[c0 + i];
                            const float t = sum[c0 + i] + y;
                            cor[c0 + i] = (t - sum[c0 + i]) - y;
                            sum[c0 + i] = t;
                        }
                    }
                    acc_release(b);
                }
#pragma unroll
                for (int i = 0; i < N; ++i) v[i] = sum[i] - cor[i];
            } else {
                (void)ks0;
                (void)ks1;
                const int b = seg % kNumAcc;
                if (acc_ready(b, (seg / kNumAcc) & 1, true)) {
#pragma unroll
                    for (int c0 = 0; c0 < N; c0 += 16) {
                        float w16[16];
                        tmem_ld16(lane_base + (uint32_t)(b * Cfg::kAccCols + c0), w16);
#pragma unroll
                        for (int i = 0; i < 16; ++i) v[c0 + i] = w16[i];
                    }
                    acc_release(b);
                } else {
                    seg_ok = false;
                }
            }
            if (!seg_ok) {
                abort_sh = 1;
                break;
            }

            const int64_t row0 = tile * kBM;
            const int64_t row = row0 + warp * 32 + lane;
            const int64_t first = sk.cta_of(tile * nk), last = sk.cta_of((tile + 1) * nk - 1);
            if (first == last) {
                // The whole K range of the tile: write it.
                store_row<N, TRANS_OUT>(v, 0, N, out, out_ld, row, M, nvalid, vec_out);
                continue;
            }
            // Shared tile.  The arrival ticket comes first: the last CTA to
            // arrive keeps its rows in registers and never writes them out
            // as a partial; every other CTA writes its partial (slot: CTA,
            // its segment index) and then counts it as written.
            unsigned int *arrived = tickets + 2 * tile, *written = arrived + 1;
            if (threadIdx.x == 0) {
                const unsigned int t = atomicAdd(arrived, 1u);
                am_last_sh = (t == (unsigned)(last - first));
            }
            epilogue_sync();
            if (!am_last_sh) {
                // Layout [N/4][128 rows] of float4: lanes write consecutive
                // 16-byte words.
                const int64_t slot = (int64_t)blockIdx.x * seg_max + orig;
                float4 *dst = reinterpret_cast<float4 *>(part + slot * (kBM * N)) + warp * 32 + lane;
#pragma unroll
                for (int i = 0; i < N; i += 4)
                    __stcg(dst + (i / 4) * kBM, make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]));
                __threadfence();
                epilogue_sync();
                if (threadIdx.x == 0) atomicAdd(written, 1u);
                continue;
            }
            // Last CTA: the others have arrived, so they are running and
            // their partials land shortly (bounded wait on the count).
            if (threadIdx.x == 0) {
                const unsigned int want =
                    (unsigned)(last - first) + (seg == segs.n - 1 ? (unsigned)g_fixup_stall : 0u);
                int ok = 0;
                for (int i = 0; i < (1 << 20); ++i) {          // ~1 s at most
                    if (atomicAdd(written, 0u) >= want) {
                        ok = 1;
                        break;
                    }
                    __nanosleep(64);
                }
                if (!ok) atomicExch(err_flag, 1);
                __threadfence();            // acquire: the partials counted above
                seg_ok_sh = ok;
            }
            epilogue_sync();
            if (!seg_ok_sh) {
                abort_sh = 1;
                break;
            }
            const int nc = (int)(last - first + 1);
            if (threadIdx.x < nc && threadIdx.x < kMaxContrib) {
                const int64_t c = first + threadIdx.x;
                contrib_sh[threadIdx.x] = (c * seg_max + (tile - sk.begin(c) / nk)) * (kBM * N);
            }
            epilogue_sync();
            // In the CTA's last segment the stage ring is idle (every stage
            // was consumed by an MMA that has completed), so the other
            // partials are fetched into it all at once (one bulk copy each,
            // one round trip) instead of one L2 round trip per contributor.
            constexpr int kTileBytes = kBM * N * (int)sizeof(float);
            const bool staged = N <= 64 && seg == segs.n - 1 && !fix_used &&
                                (int64_t)(nc - 1) * kTileBytes <= (int64_t)kStages * Cfg::kStageBytes;
            if (staged && nc <= kMaxContrib) {
                if (threadIdx.x == 0) {
                    // Generic-proxy writes of the other CTAs (acquired above)
                    // before the async-proxy reads below.
                    asm volatile("fence.proxy.async;" ::: "memory");
                    mbar_expect_tx(&fix_bar, (uint32_t)((nc - 1) * kTileBytes));
                    for (int j = 0, q = 0; j < nc; ++j)
                        if (first + j != (int64_t)blockIdx.x)
                            bulk_load(smem + (q++) * kTileBytes, part + contrib_sh[j], kTileBytes,
                                      &fix_bar);
                }
                if (threadIdx.x == 64) seg_ok_sh = mbar_wait(&fix_bar, 0, err_flag);
                epilogue_sync();
                const int fetched = seg_ok_sh;
                epilogue_sync();
                fix_used = true;
                if (!fetched) {
                    abort_sh = 1;
                    break;
                }
            }
            if (nc > kMaxContrib) {
                if (threadIdx.x == 0) atomicExch(err_flag, 2);
            } else if (N <= 64 && staged) {
                // Same order and arithmetic as below, from shared memory.
                const float4 *stg = reinterpret_cast<const float4 *>(smem) + warp * 32 + lane;
                float sum[N];
#pragma unroll
                for (int i = 0; i < N; ++i) sum[i] = 0.0f;
                for (int j = 0, q = 0; j < nc; ++j) {
                    if (first + j == (int64_t)blockIdx.x) {
#pragma unroll
                        for (int i = 0; i < N; ++i) sum[i] += v[i];
                    } else {
                        const float4 *src = stg + (int64_t)(q++) * (kTileBytes / 16);
#pragma unroll
                        for (int i = 0; i < N / 4; ++i) {
                            const float4 w = src[i * kBM];
                            sum[4 * i] += w.x;
                            sum[4 * i + 1] += w.y;
                            sum[4 * i + 2] += w.z;
                            sum[4 * i + 3] += w.w;
                        }
                    }
                }
                store_row<N, TRANS_OUT>(sum, 0, N, out, out_ld, row, M, nvalid, vec_out);
            } else {
                // The sum runs in CTA order whichever CTA is last
                // (deterministic).  Up to 64 columns a thread loads a whole
                // partial row at once (one L2 round trip per contributor);
                // wider tiles go in column blocks of 16 to bound registers.
                constexpr int CB = N <= 64 ? N : 16;
#pragma unroll
                for (int cb = 0; cb < N; cb += CB) {
                    float sum[CB];
#pragma unroll
                    for (int i = 0; i < CB; ++i) sum[i] = 0.0f;
                    for (int j = 0; j < nc; ++j) {
                        if (first + j == (int64_t)blockIdx.x) {
#pragma unroll
                            for (int i = 0; i < CB; ++i) sum[i] += v[cb + i];
                        } else {
                            const float4 *src = reinterpret_cast<const float4 *>(
                                                    part + contrib_sh[j]) +
                                                (cb / 4) * kBM + warp * 32 + lane;
                            float4 w[CB / 4];
#pragma unroll
                            for (int i = 0; i < CB / 4; ++i) w[i] = __ldcg(src + i * kBM);
#pragma unroll
                            for (int i = 0; i < CB / 4; ++i) {
                                sum[4 * i] += w[i].x;
                                sum[4 * i + 1] += w[i].y;
                                sum[4 * i + 2] += w[i].z;
                                sum[4 * i + 3] += w[i].w;
                            }
                        }
                    }
                    store_row<CB, TRANS_OUT>(sum, cb, N, out, out_ld, row, M, nvalid, vec_out);
                }
            }
            if (threadIdx.x == 0) {
                arrived[0] = 0u;
                written[0] = 0u;
            }
        }
    }

    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(Cfg::kTmemCols)
                     : "memory");
    }
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
    int64_t tiles;
    int nk, grid, seg_max;
};

// One persistent CTA per SM (the stage ring fills most of its shared
// memory), each with an equal share of the (row tile, K stage) units.
template <int KIND, int N>
TcPlan plan_for(int64_t M, int64_t K) {
    using Cfg = TcCfg<KIND, N>;
    TcPlan p;
    p.tiles = (M + kBM - 1) / kBM;
    p.nk = (int)((K + Cfg::kBK - 1) / Cfg::kBK);
    const int64_t total = p.tiles * p.nk;
    p.grid = (int)(total < kNumSMs ? total : kNumSMs);
    // At most 32 CTAs per row tile keeps a tile's contributors <= 34 < kMaxContrib.
    if (p.grid > p.tiles * 32) p.grid = (int)(p.tiles * 32);
    const int64_t per = p.grid > 0 ? (total + p.grid - 1) / p.grid : 0;
    p.seg_max = p.nk > 0 ? (int)((per + p.nk - 1) / p.nk + 1) : 1;
    return p;
}

template <int KIND, int N, bool TRANS>
cudaError_t tc_launch(const TcOperands &o, float *out, int64_t out_ld, void *ws,
                      unsigned int *tickets, int *err_flag, cudaStream_t st) {
    using Cfg = TcCfg<KIND, N>;
    const TcPlan p = plan_for<KIND, N>(o.M, o.K);
    if (p.grid < 1) return cudaErrorInvalidValue;
    CUtensorMap mq, mql;
    const bool bf = KIND == 1;
    // Q has q_rows <= N real rows; the N-row box reads zeros beyond them.
    if (!make_map(&mq, o.Q, bf, o.q_rows, o.K, o.ldq, N)) return cudaErrorInvalidValue;
    if (bf) {
        if (!make_map(&mql, o.Q_lo, bf, o.q_rows, o.K, o.ldq, N)) return cudaErrorInvalidValue;
    } else {
        mql = mq;
    }
    const size_t smem = (size_t)Cfg::kStages * Cfg::kStageBytes + 1024;
    auto kern = tc_gemm_kernel<KIND, N, TRANS>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    // Programmatic dependent launch: the kernel may begin while the
    // preceding kernel in the stream still runs (it waits for it before the
    // first read of Q, see the producer).
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)p.grid);
    cfg.blockDim = dim3(kTcThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = o.no_pdl ? 0 : 1;
    return cudaLaunchKernelEx(&cfg, kern, static_cast<const unsigned char *>(o.P),
                              static_cast<const unsigned char *>(o.P_lo), mq, mql, o.M, p.tiles,
                              p.nk, o.nvalid, out, out_ld, static_cast<float *>(ws), p.seg_max,
                              tickets, err_flag);
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

// Packed P: for every 128-row tile t and 128-byte K atom a, one 16 KiB block
// at ((t * atoms + a) * 16 KiB) that is the exact shared-memory image a TMA
// load with 128-byte swizzle would produce: row i at i * 128 bytes, its
// 16-byte chunk c at chunk position c ^ (i % 8).  Rows >= M and K >= K are
// zero.  `atoms` is the number of atoms per tile, a whole number of stages.
// TF32: 32 fp32 per atom row.  BF16X3: 64 bf16 per atom row, in a hi and a
// lo array (x ~ hi + lo).
template <bool TRANS, bool BF>
__global__ void __launch_bounds__(256)
pack_kernel(const float *__restrict__ x, int64_t rows, int64_t cols, int64_t ld, int64_t atoms,
            unsigned char *__restrict__ out_hi, unsigned char *__restrict__ out_lo) {
    // P = x (TRANS false: M = rows, K = cols) or P = x^T (M = cols, K = rows).
    constexpr int kAtomK = BF ? 64 : 32;
    const int64_t M = TRANS ? cols : rows, K = TRANS ? rows : cols;
    const int64_t t = blockIdx.y, a = blockIdx.x;
    __shared__ float tile[TRANS ? kAtomK : 1][TRANS ? 129 : 1];
    if constexpr (TRANS) {
        // Stage x[a*kAtomK .. +kAtomK][t*128 .. +128] (coalesced along columns).
        for (int e = threadIdx.x; e < kAtomK * 128; e += 256) {
            const int kr = e / 128, ci = e % 128;
            const int64_t gr = a * kAtomK + kr, gc = t * 128 + ci;
            tile[kr][ci] = (gr < rows && gc < cols) ? x[gr * ld + gc] : 0.0f;
        }
        __syncthreads();
    }
    unsigned char *blk_hi = out_hi + (t * atoms + a) * 16384;
    unsigned char *blk_lo = BF ? out_lo + (t * atoms + a) * 16384 : nullptr;
    constexpr int kPer = BF ? 8 : 4;                 // elements per 16-byte chunk
    for (int e = threadIdx.x; e < 128 * 8; e += 256) {
        const int i = e / 8, c = e % 8;              // P row in the tile, chunk
        const int64_t prow = t * 128 + i;
        float v[kPer];
#pragma unroll
        for (int j = 0; j < kPer; ++j) {
            const int64_t k = a * kAtomK + c * kPer + j;
            if constexpr (TRANS) v[j] = tile[c * kPer + j][i];
            else v[j] = (prow < M && k < K) ? x[prow * ld + k] : 0.0f;
        }
        const int pos = i * 128 + ((c ^ (i & 7)) << 4);
        if constexpr (BF) {
            __align__(16) __nv_bfloat16 h[8], l[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                h[j] = __float2bfloat16_rn(v[j]);
                l[j] = __float2bfloat16_rn(v[j] - __bfloat162float(h[j]));
            }
            *reinterpret_cast<uint4 *>(blk_hi + pos) = *reinterpret_cast<const uint4 *>(h);
            *reinterpret_cast<uint4 *>(blk_lo + pos) = *reinterpret_cast<const uint4 *>(l);
        } else {
            *reinterpret_cast<float4 *>(blk_hi + pos) =
                make_float4(tf32_rna(v[0]), tf32_rna(v[1]), tf32_rna(v[2]), tf32_rna(v[3]));
        }
    }
}

// The factor operand of a tensor-core product as the tensor cores see it.
// TF32: q = tf32_rna(x).  BF16X3: hi = bf16(x), lo = bf16(x - hi) and
// q = hi + lo.  The Gram of the same factor is then formed from q, so that
// the product, the Gram and the Remark 1 error they feed all refer to one
// matrix; with the product and the Gram rounded differently the error
// carries a random term of about u ||X||^2 / sqrt(r n) per iteration (u
// the operand rounding), far above the differences the restart test has
// to resolve near convergence.
template <bool BF>
__device__ __forceinline__ float operand_value(float x, __nv_bfloat16 &h, __nv_bfloat16 &l) {
    if constexpr (BF) {
        h = __float2bfloat16_rn(x);
        l = __float2bfloat16_rn(x - __bfloat162float(h));
        return __bfloat162float(h) + __bfloat162float(l);
    } else {
        return tf32_rna(x);
    }
}

// Element-wise over rows x cols (row stride ld; H_y is r x ld): q, and for
// BF16X3 the hi / lo arrays, in the same layout.
template <bool BF>
__global__ void __launch_bounds__(256)
prep_h_kernel(const float *__restrict__ x, int64_t rows, int64_t cols, int64_t ld,
              float *__restrict__ q, __nv_bfloat16 *__restrict__ hi,
              __nv_bfloat16 *__restrict__ lo) {
    // Lets a programmatically dependent product kernel start its X stream.
    asm volatile("griddepcontrol.launch_dependents;");
    const int64_t count = rows * cols;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = (e / cols) * ld + e % cols;
        __nv_bfloat16 h, l;
        q[i] = operand_value<BF>(x[i], h, l);
        if constexpr (BF) {
            hi[i] = h;
            lo[i] = l;
        }
    }
}

// W_y (rows x cols, row stride ld_in): q in the same layout (for the Gram),
// and the transposed operand (cols x rows, row stride ld_t): q^T for TF32,
// hi^T / lo^T for BF16X3.
template <bool BF>
__global__ void prep_w_kernel(const float *__restrict__ x, int64_t rows, int64_t cols,
                              int64_t ld_in, float *__restrict__ q, float *__restrict__ qt,
                              __nv_bfloat16 *__restrict__ ht, __nv_bfloat16 *__restrict__ lt,
                              int64_t ld_t) {
    asm volatile("griddepcontrol.launch_dependents;");
    __shared__ float tq[32][33];
    __shared__ __nv_bfloat16 th[32][34], tl[32][34];
    const int64_t r0 = (int64_t)blockIdx.x * 32, c0 = (int64_t)blockIdx.y * 32;
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
        const int64_t rr = r0 + y, cc = c0 + threadIdx.x;
        float v = 0.0f;
        __nv_bfloat16 h = __float2bfloat16_rn(0.0f), l = h;
        if (rr < rows && cc < cols) {
            v = operand_value<BF>(x[rr * ld_in + cc], h, l);
            q[rr * ld_in + cc] = v;
        }
        tq[y][threadIdx.x] = v;
        th[y][threadIdx.x] = h;
        tl[y][threadIdx.x] = l;
    }
    __syncthreads();
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
        const int64_t cc = c0 + y, rr = r0 + threadIdx.x;
        if (cc < cols && rr < rows) {
            if constexpr (BF) {
                ht[cc * ld_t + rr] = th[threadIdx.x][y];
                lt[cc * ld_t + rr] = tl[threadIdx.x][y];
            } else {
                qt[cc * ld_t + rr] = tq[threadIdx.x][y];
            }
        }
    }
}

}  // namespace

cudaError_t launch_tc_prep_h(const float *H, int64_t rows, int64_t cols, int64_t ld,
                             int precision, float *q, __nv_bfloat16 *hi, __nv_bfloat16 *lo,
                             cudaStream_t st) {
    int64_t blocks = (rows * cols + 255) / 256;
    if (blocks > 4 * kNumSMs) blocks = 4 * kNumSMs;
    if (blocks < 1) blocks = 1;
    if (precision == NMF_PREC_TF32)
        prep_h_kernel<false><<<(unsigned)blocks, 256, 0, st>>>(H, rows, cols, ld, q, hi, lo);
    else if (precision == NMF_PREC_BF16X3)
        prep_h_kernel<true><<<(unsigned)blocks, 256, 0, st>>>(H, rows, cols, ld, q, hi, lo);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t launch_tc_prep_w(const float *W, int64_t rows, int64_t cols, int64_t ld_in,
                             int precision, float *q, float *qt, __nv_bfloat16 *ht,
                             __nv_bfloat16 *lt, int64_t ld_t, cudaStream_t st) {
    dim3 grid((unsigned)((rows + 31) / 32), (unsigned)((cols + 31) / 32));
    if (grid.y > 65535) return cudaErrorInvalidValue;
    if (precision == NMF_PREC_TF32)
        prep_w_kernel<false><<<grid, dim3(32, 8), 0, st>>>(W, rows, cols, ld_in, q, qt, ht, lt, ld_t);
    else if (precision == NMF_PREC_BF16X3)
        prep_w_kernel<true><<<grid, dim3(32, 8), 0, st>>>(W, rows, cols, ld_in, q, qt, ht, lt, ld_t);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

template <int KIND>
TcPlan plan_dispatch(int64_t M, int64_t K, int N) {
    switch (N) {
        case 16: return plan_for<KIND, 16>(M, K);
        case 32: return plan_for<KIND, 32>(M, K);
        case 48: return plan_for<KIND, 48>(M, K);
        case 64: return plan_for<KIND, 64>(M, K);
        case 80: return plan_for<KIND, 80>(M, K);
        case 96: return plan_for<KIND, 96>(M, K);
        case 112: return plan_for<KIND, 112>(M, K);
        default: return plan_for<KIND, 128>(M, K);
    }
}

size_t tc_ws_bytes(int64_t M, int64_t K, int N, int precision) {
    const TcPlan p = precision == NMF_PREC_TF32 ? plan_dispatch<0>(M, K, N)
                                                : plan_dispatch<1>(M, K, N);
    return sizeof(float) * (size_t)(p.grid > 0 ? p.grid : 1) * p.seg_max * kBM * N;
}

// Two counters per row tile: CTAs arrived, partials written.
int64_t tc_num_tickets(int64_t M) { return 2 * ((M + kBM - 1) / kBM); }

// Atoms per tile of the packed P: K rounded up to whole stages.
int64_t tc_packed_atoms(int64_t K, int precision) {
    const int bk = 64;                               // K elements per stage, both precisions
    const int atoms_per_stage = precision == NMF_PREC_TF32 ? 2 : 1;
    return (K + bk - 1) / bk * atoms_per_stage;
}

size_t tc_packed_bytes(int64_t M, int64_t K, int precision) {
    return (size_t)((M + kBM - 1) / kBM) * (size_t)tc_packed_atoms(K, precision) * 16384;
}

cudaError_t launch_tc_pack(const float *x, int64_t rows, int64_t cols, int64_t ld, bool transposed,
                           int precision, void *out_hi, void *out_lo, cudaStream_t st) {
    const int64_t M = transposed ? cols : rows, K = transposed ? rows : cols;
    const int64_t atoms = tc_packed_atoms(K, precision);
    const int64_t tiles = (M + kBM - 1) / kBM;
    if (tiles > 65535 || atoms > 0x7fffffff) return cudaErrorInvalidValue;
    dim3 grid((unsigned)atoms, (unsigned)tiles);
    auto *hi = static_cast<unsigned char *>(out_hi);
    auto *lo = static_cast<unsigned char *>(out_lo);
    if (precision == NMF_PREC_TF32) {
        if (transposed) pack_kernel<true, false><<<grid, 256, 0, st>>>(x, rows, cols, ld, atoms, hi, lo);
        else pack_kernel<false, false><<<grid, 256, 0, st>>>(x, rows, cols, ld, atoms, hi, lo);
    } else if (precision == NMF_PREC_BF16X3) {
        if (transposed) pack_kernel<true, true><<<grid, 256, 0, st>>>(x, rows, cols, ld, atoms, hi, lo);
        else pack_kernel<false, true><<<grid, 256, 0, st>>>(x, rows, cols, ld, atoms, hi, lo);
    } else {
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

bool tc_available() { return encode_fn() != nullptr; }

cudaError_t tc_set_fixup_stall(int extra) {
    return cudaMemcpyToSymbol(g_fixup_stall, &extra, sizeof(int));
}

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

}  // namespace nmfg
