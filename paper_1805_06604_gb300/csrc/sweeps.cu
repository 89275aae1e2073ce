// sweeps.cu -- A-HALS inner loops on H (Sec. 1 of Ang & Gillis, arXiv
// 1805.06604) as a blocked Gauss-Seidel with a chain warp and product warps.
//
// For every column j of H independently, `sweeps` cyclic passes of
//   H(k,j) <- max(0, (A(k,j) - sum_{i != k} G(k,i) H(i,j)) / G(k,k)),
// k = 0..r-1, with A = W_y^T X and G = W_y^T W_y (the W side, many more
// items, runs the lane-pipelined kernel of hals_impl.cuh).  A zero G(k,k)
// leaves the coordinate unchanged (the paper does not treat it; the whole
// k-th Gram row is then zero, so the coordinate enters no other update).
//
// Work decomposition.  A CTA owns up to 32 items (columns of H); their
// iterates x (RP x 32, RP = r rounded up to a multiple of B = 8,
// padding coordinates have a zero Gram row and column and stay zero), the
// right-hand sides a and the Gram live in shared memory for all sweeps.
// The coordinates are cut into blocks K_b of B consecutive ones.  The sum of
// update k in K_b splits into
//
//   s_k = [a_k - sum_{i not in K_{b-1} u K_b} G(k,i) x_i]          P_b(k)
//         - sum_{i in K_{b-1}} G(k,i) x_i                           fold-in
//         - sum_{i in K_b, i != k} G(k,i) x_i                       in block
//
// (blocks cyclic: K_{-1} is the last block, updated at the end of the
// previous sweep).  P_b only reads coordinates that are final before block
// b-1 starts, so the three product warps compute it for all 32 items while
// the chain warp runs block b-1: one lane per item, the B updates of a block
// in sequence, each in the paper's dot-product form from the current
// iterate (so no rounding accumulates across sweeps).  The warps hand
// blocks over through named barriers, two buffers deep:
//   P-ready(g):  product warps arrive after writing P of global block g,
//                the chain warp waits before block g (ids 1, 2 by parity);
//   X-ready(g):  the chain warp arrives after storing block g's new values,
//                the product warps wait before P of block g + 2 (ids 3, 4).
// The sequence of updates is exactly the cyclic order of the paper; only
// the order in which each sum is accumulated differs.
//
// Fused epilogue (after the sweeps): H_y = H_n + beta (H_n - H) (projected
// for hp = 3), Algorithm 2 steps 4-9.
#include <cuda_runtime.h>
#include <math.h>

#include "common.cuh"
#include "decide.cuh"

namespace nmfg {
namespace {

constexpr int kItems = 32;            // items per CTA: one per lane of the chain warp
constexpr int kThreads = 128;         // warp 0: chain; warps 1-3: block products
constexpr int kProdWarps = 3;

enum ItemLayout { kColumn = 0, kRow = 1 };

template <int L>
__device__ __forceinline__ int64_t elem_index(int64_t item, int k, int64_t ld) {
    return L == kColumn ? (int64_t)k * ld + item : item * ld + k;
}

// Named barriers with immediate ids (so the CTA reserves only ids 0-4):
// id0 + parity selects one of a pair.
template <int ID0>
__device__ __forceinline__ void bar_sync(int parity) {
    if (parity) asm volatile("bar.sync %0, %1;" ::"n"(ID0 + 1), "n"(kThreads) : "memory");
    else asm volatile("bar.sync %0, %1;" ::"n"(ID0), "n"(kThreads) : "memory");
}
template <int ID0>
__device__ __forceinline__ void bar_arrive(int parity) {
    if (parity) asm volatile("bar.arrive %0, %1;" ::"n"(ID0 + 1), "n"(kThreads) : "memory");
    else asm volatile("bar.arrive %0, %1;" ::"n"(ID0), "n"(kThreads) : "memory");
}

__device__ __forceinline__ float4 lds4(const float *p) {
    return *reinterpret_cast<const float4 *>(p);
}


// Shared-memory carve-up (in floats; every part 16-byte aligned).
struct Layout {
    int rp, rps;             // padded coordinates; item row stride of x and a (rp + 4)
    int g, x, a, p, inv, total;
    __host__ __device__ Layout(int r, int B) {
        rp = (r + B - 1) / B * B;
        rp = (rp + 3) / 4 * 4;
        rps = rp + 4;        // (rp + 4) / 4 is odd: 16-byte loads of 8 lanes hit 8 banks
        g = 0;                               // G[k][i], rp x rp
        x = g + rp * rp;                     // x[item][k], 32 x rps
        a = x + kItems * rps;                // a[item][k], 32 x rps
        p = a + kItems * rps;                // P[buf][warp][item][B], 2 x 3 x 32 x B
        inv = p + 2 * kProdWarps * kItems * B;   // 1 / G(k,k) or 0, rp
        total = inv + rp;
    }
};

template <int B>
__device__ __forceinline__ void ld_vec(float (&v)[B], const float *p) {
#pragma unroll
    for (int q = 0; q < B; q += 4) {
        const float4 u = lds4(p + q);
        v[q] = u.x;
        v[q + 1] = u.y;
        v[q + 2] = u.z;
        v[q + 3] = u.w;
    }
}
template <int B>
__device__ __forceinline__ void st_vec(float *p, const float (&v)[B]) {
#pragma unroll
    for (int q = 0; q < B; q += 4)
        *reinterpret_cast<float4 *>(p + q) = make_float4(v[q], v[q + 1], v[q + 2], v[q + 3]);
}

template <int LAYOUT, int B>
__device__ __forceinline__ void
sweep_body(int64_t items, int r, int64_t ld, int nt,
           const float *__restrict__ Aglob,     // right-hand side a (A or C)
           const float *__restrict__ Gglob,     // Gram (G or D), rs x rs
           int rs, const float *Xin, float *Xout, int sweeps,   // may alias (one sweep in place)
           const HEpilogue &hep, int64_t bid) {
    // A programmatically dependent successor (the tensor-core X product)
    // may start streaming X now; it waits for this grid before reading H_y.
    asm volatile("griddepcontrol.launch_dependents;");
    extern __shared__ __align__(16) float smem[];
    const Layout L(r, B);
    const int rp = L.rp, rps = L.rps, nb = rp / B;
    float *Gs = smem + L.g, *xs = smem + L.x, *as = smem + L.a, *Pb = smem + L.p;
    float *inv = smem + L.inv;
    const int64_t item0 = bid * nt;
    const int nhere = (int)(items - item0 < (int64_t)nt ? items - item0 : (int64_t)nt);
    const int tid = threadIdx.x, lane = tid % 32, warp = tid / 32;
    __shared__ double sh32[32];
    if (sweep_stopped(hep.stop, sh32, bid)) return;    // A-HALS early stop (delta rule)

    for (int e = tid; e < rp * rp; e += kThreads) {
        const int k = e / rp, i = e % rp;
        Gs[e] = (k < r && i < r) ? Gglob[k * rs + i] : 0.0f;
    }
    for (int k = tid; k < rp; k += kThreads) {
        const float d = k < r ? Gglob[k * rs + k] : 0.0f;
        inv[k] = d > 0.0f ? 1.0f / d : 0.0f;
    }
    // Coalesced global reads: consecutive threads take consecutive items of
    // one coordinate (H side) or consecutive coordinates of one item (W side).
    for (int e = tid; e < rp * kItems; e += kThreads) {
        int k, j;
        if (LAYOUT == kColumn) {
            k = e / kItems;
            j = e % kItems;
        } else {
            j = e / rp;
            k = e % rp;
        }
        const bool in = j < nhere && k < r;
        const int64_t q = in ? elem_index<LAYOUT>(item0 + j, k, ld) : 0;
        xs[j * rps + k] = in ? Xin[q] : 0.0f;
        as[j * rps + k] = in ? Aglob[q] : 0.0f;
    }
    __syncthreads();

    const int total = sweeps * nb;
    if (warp == 0) {
        // ------------------------------------------------ chain warp
        // Registers carry, into block g: gin (G of the block with itself),
        // iv (1 / G(k,k)), xc (the block's values before the update), corr
        // (the fold-in of the previous block's new values) and old (the
        // in-block sums over the coordinates after k, from old values).
        float *xrow = xs + lane * rps;
        float gin[B][B], iv[B], xc[B], corr[B], old[B];
        auto prefetch = [&](int b, const float (&xnew)[B], int bprev) {
            // Block b's tiles; its fold-in from block bprev's new values.
#pragma unroll
            for (int kb = 0; kb < B; ++kb) ld_vec<B>(gin[kb], Gs + (b * B + kb) * rp + b * B);
            ld_vec<B>(iv, inv + b * B);
            ld_vec<B>(xc, xrow + b * B);
#pragma unroll
            for (int kb = 0; kb < B; ++kb) {
                float gf[B];
                ld_vec<B>(gf, Gs + (b * B + kb) * rp + bprev * B);
                float t0 = 0.0f, t1 = 0.0f;
#pragma unroll
                for (int q = 0; q < B; q += 2) {
                    t0 = fmaf(-gf[q], xnew[q], t0);
                    t1 = fmaf(-gf[q + 1], xnew[q + 1], t1);
                }
                corr[kb] = nb > 1 ? t0 + t1 : 0.0f;
                float o = 0.0f;
#pragma unroll
                for (int q = kb + 1; q < B; ++q) o = fmaf(-gin[kb][q], xc[q], o);
                old[kb] = o;
            }
        };
        {
            float xl[B];
            ld_vec<B>(xl, xrow + (nb - 1) * B);
            prefetch(0, xl, nb - 1);
        }
        int b = 0;
#pragma unroll 1
        for (int g = 0; g < total; ++g) {
            const int buf = g & 1;
            bar_sync<1>(buf);                                // P of block g is ready
            float y[B];
            {
                float p0[B], p1[B], p2[B];
                const float *pb = Pb + (buf * kProdWarps * kItems + lane) * B;
                ld_vec<B>(p0, pb);
                ld_vec<B>(p1, pb + kItems * B);
                ld_vec<B>(p2, pb + 2 * kItems * B);
#pragma unroll
                for (int kb = 0; kb < B; ++kb) y[kb] = ((p0[kb] + p1[kb]) + (p2[kb] + corr[kb])) + old[kb];
            }
            // The B updates of the block, in order: the terms of values new
            // in this block are added last, the newest one last of all.
#pragma unroll
            for (int kb = 0; kb < B; ++kb) {
                float s = y[kb];
#pragma unroll
                for (int q = 0; q < kb; ++q) s = fmaf(-gin[kb][q], xc[q], s);
                const float h = fmaxf(s * iv[kb], 0.0f);
                if (iv[kb] > 0.0f) xc[kb] = h;
            }
            st_vec<B>(xrow + b * B, xc);
            bar_arrive<3>(buf);                              // block g's values are stored
            const int bn = b + 1 == nb ? 0 : b + 1;
            {
                float xnew[B];
#pragma unroll
                for (int q = 0; q < B; ++q) xnew[q] = xc[q];
                prefetch(bn, xnew, b);
            }
            b = bn;
        }
    } else {
        // ------------------------------------------------ product warps
        // For block b, P(k) = a_k - sum G(k,i) x_i over the blocks other than
        // b-1 and b; warp w (0..2) sums every third of those blocks (in the
        // cyclic order b+1, b+2, ...) for all B rows and its 32 items, and
        // warp 0 starts from a_k.  The chain warp adds the three partials.
        const int w = warp - 1;
        const float *xrow = xs + lane * rps;
        int b = 0;
#pragma unroll 1
        for (int g = 0; g < total; ++g) {
            const int buf = g & 1;
            if (g >= 2) bar_sync<3>(buf);                    // block g-2 is stored
            float acc[B];
            if (w == 0) ld_vec<B>(acc, as + lane * rps + b * B);
            else {
#pragma unroll
                for (int kb = 0; kb < B; ++kb) acc[kb] = 0.0f;
            }
            // B independent row sums: each block adds a chain of B FMAs per
            // row, and the B rows interleave to cover the FMA latency.
            const float *grow = Gs + b * B * rp;
            int c = b + 1 + w;                               // block b+1+w, then every third
            if (c >= nb) c -= nb;
#pragma unroll 1
            for (int q = 1 + w; q <= nb - 2; q += kProdWarps) {
                float xv[B];
                ld_vec<B>(xv, xrow + c * B);
#pragma unroll
                for (int kb = 0; kb < B; ++kb) {
                    float gv[B];
                    ld_vec<B>(gv, grow + kb * rp + c * B);
#pragma unroll
                    for (int u = 0; u < B; ++u) acc[kb] = fmaf(-gv[u], xv[u], acc[kb]);
                }
                c += kProdWarps;
                if (c >= nb) c -= nb;
            }
            st_vec<B>(Pb + ((buf * kProdWarps + w) * kItems + lane) * B, acc);
            bar_arrive<1>(buf);                              // P of block g is ready
            b = b + 1 == nb ? 0 : b + 1;
        }
        // The last two blocks' stores have not been waited for yet.
        for (int g = total - 2 < 0 ? 0 : total - 2; g < total; ++g) bar_sync<3>(g & 1);
    }
    __syncthreads();

    // ---------------------------------------------------- results
    double moved = 0.0;                                 // ||change||^2 (delta rule)
    for (int e = tid; e < rp * kItems; e += kThreads) {
        int k, j;
        if (LAYOUT == kColumn) {
            k = e / kItems;
            j = e % kItems;
        } else {
            j = e / rp;
            k = e % rp;
        }
        if (j < nhere && k < r) {
            const int64_t q = elem_index<LAYOUT>(item0 + j, k, ld);
            const float x = xs[j * rps + k];
            if (hep.stop.l > 0) {
                const double dx = (double)x - (double)Xin[q];
                moved = fma(dx, dx, moved);
            }
            Xout[q] = x;
            if (LAYOUT == kColumn && hep.Hw != nullptr) {
                // Algorithm 2 steps 4-9: H_y = H_n + beta (H_n - H), projected if hp = 3.
                const float beta = (float)hep.state->beta;
                float v = fmaf(beta, x - hep.H_acc[q], x);
                if (hep.hp == 3) v = fmaxf(v, 0.0f);
                hep.Hw[q] = v;
            }
        }
    }
    sweep_record(hep.stop, moved, sh32, bid);

}

template <int LAYOUT, int B>
__global__ void __launch_bounds__(kThreads)
sweep_kernel(int64_t items, int r, int64_t ld, int nt, const float *__restrict__ Aglob,
             const float *__restrict__ Gglob, int rs, const float *Xin, float *Xout, int sweeps,
             HEpilogue hep) {
    sweep_body<LAYOUT, B>(items, r, ld, nt, Aglob, Gglob, rs, Xin, Xout, sweeps, hep, blockIdx.x);
}
template <int LAYOUT, int B>
__global__ void __launch_bounds__(kThreads)
sweep_grouped(const SweepItem *__restrict__ table, const int64_t *__restrict__ begin,
              int nitems) {
    int64_t local;
    const SweepItem &it = table[group_item(begin, nitems, local)];
    sweep_body<LAYOUT, B>(it.items, it.r, it.ld, it.nt, it.A, it.G, it.rs, it.Xin, it.Xout,
                          it.sweeps, it.hep, local);
}

// Coordinates per block.  Each block costs one hand-over between the
// chain warp and the product warps (about 200 cycles of barrier round trip
// on GB300, measured), and the chain warp about 2B + 6 instructions per
// update; B = 8 measured fastest on the dense 10000 x 4000 r = 50 and
// 10304 x 4000 r = 64 workloads (B = 4: 413 / 452 us, B = 8: 260 / 256 us
// for the H side).
constexpr int kBlockH = 8;

// Items per CTA: 32, one per lane of the chain warp.  A CTA's time is set
// by its chain warp whatever its item count, so full CTAs leave the most SMs
// to other work (the batched solver runs many instances side by side; dense
// 4000 columns: 125 CTAs of 32 take as long as 149 of 27).
int items_per_cta(int64_t items) {
    (void)items;
    return kItems;
}

template <int LAYOUT, int B>
cudaError_t sweep_launch(int64_t items, int r, int64_t ld, const float *A, const float *G, int rs,
                         const float *Xin, float *Xout, int sweeps, const HEpilogue &hep,
                         cudaStream_t st) {
    const Layout L(r, B);
    const size_t smem = sizeof(float) * (size_t)L.total;
    auto kern = sweep_kernel<LAYOUT, B>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    const int nt = items_per_cta(items);
    const unsigned grid = (unsigned)((items + nt - 1) / nt);
    if (grid == 0) return cudaSuccess;
    kern<<<grid, kThreads, smem, st>>>(items, r, ld, nt, A, G, rs, Xin, Xout, sweeps, hep);
    return cudaGetLastError();
}

}  // namespace

int hals_h_num_ctas(int64_t n, int r) {
    (void)r;
    const int nt = items_per_cta(n);
    return (int)((n + nt - 1) / nt);
}

cudaError_t launch_hals_h(int64_t n, int64_t ldh, int r, int rs, const float *A,
                          const float *G, const float *H_in, float *H_out, int sweeps,
                          const HEpilogue &ep, cudaStream_t st) {
    return sweep_launch<kColumn, kBlockH>(n, r, ldh, A, G, rs, H_in, H_out, sweeps, ep, st);
}


// ------------------------------------------------------------ grouped launches
// The H sweeps of many problems in one launch.  The columns per CTA (nt <=
// 32; 0: the single launch's choice) set only how the columns are grouped
// into CTAs: every column's updates are the same whatever the grouping.
void plan_sweep_h_item(int64_t n, int64_t ldh, int r, int rs, const float *A, const float *G,
                       const float *H_in, float *H_out, int sweeps, const HEpilogue &ep, int nt,
                       SweepItem *it, int64_t *ctas) {
    if (nt <= 0 || nt > kItems) nt = items_per_cta(n);
    *it = SweepItem{n, r, ldh, nt, A, G, rs, H_in, H_out, sweeps, ep};
    *ctas = (n + nt - 1) / nt;
}

cudaError_t launch_sweep_h_grouped(const SweepItem *items, const int64_t *begin, int nitems,
                                   int64_t ctas, int max_r, cudaStream_t st) {
    if (nitems < 1 || ctas < 1) return cudaSuccess;
    const Layout L(max_r, kBlockH);
    const size_t smem = sizeof(float) * (size_t)L.total;
    auto kern = sweep_grouped<kColumn, kBlockH>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)ctas, kThreads, smem, st>>>(items, begin, nitems);
    return cudaGetLastError();
}

}  // namespace nmfg
