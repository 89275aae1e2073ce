// hals_rows.cu -- dispatch of the lane-pipelined A-HALS sweep kernel
// (hals_impl.cuh) on the rows of W: picks the lanes per item T and the
// smallest instantiated slot count S >= ceil(r/T).  (The H side runs the
// blocked kernel of sweeps.cu.)
#include "common.cuh"

namespace nmfg {

template <int T, int S, int LAYOUT>
cudaError_t hals_launch(int64_t items, int r, int64_t ld, const float *A, const float *G, int rs,
                        const float *Xin, float *Xout, int sweeps, const HEpilogue &hep,
                        const WEpilogue &wep, int cta_threads, cudaStream_t st);

template <int T, int S>
cudaError_t hals_w_launch_grouped(const HalsWItem *items, const int64_t *begin, int nitems,
                                  int64_t ctas, int cta_threads, cudaStream_t st);

namespace {

// Two lanes per item up to r = 64, four lanes above (r <= 128): every slot
// count is instantiated so that an item is padded by less than T coordinates.
constexpr int kSlots4[] = {17, 18, 19, 20, 21, 22, 23, 24, 25, 26, 27, 28, 29, 30, 31, 32};
constexpr int kSlots2[] = {2,  3,  4,  5,  6,  7,  8,  9,  10, 11, 12, 13, 14, 15, 16, 17,
                           18, 19, 20, 21, 22, 23, 24, 25, 26, 27, 28, 29, 30, 31, 32};
// Threads per CTA of a sweep launch.  Between ~0.4 and two warps per
// scheduler of the GPU, 96-thread CTAs (three warps) spread the warps over
// more SMs than 128-thread ones and leave fewer SMs with a double share than
// 64-thread ones (dense 10000 x 4000 r = 50: H side 250 warps 342.7 us
// against 347.5 at 128; W side 625 warps 180.7 us against 184.2 at 64 and
// 200 at 128).  Outside that range -- the small, batched and sparse
// problems -- 128 measured best.
int cta_threads(int64_t items, int T) {
    const int64_t warps = (items * T + 31) / 32;
    const int64_t schedulers = 4LL * kNumSMs;
    return (warps * 5 >= 2 * schedulers && warps <= 2 * schedulers) ? 96 : 128;
}

template <int N>
int pick(const int (&list)[N], int need) {
    for (int v : list)
        if (v >= need) return v;
    return -1;
}

// Lanes per item.  The time of a sweep is set by the latency of one update
// of an item, which grows with T (longer butterfly and chain), while the
// items of all warps run concurrently; so the smallest T whose registers
// hold the item wins -- measured on the dense 10000 x 4000 r = 50 and the
// 2000 x 1500 r = 24 problems, T = 2 beat T = 4 and T = 8 on both sides.
int pick_lanes(int r) { return r <= 64 ? 2 : 4; }

template <int LAYOUT>
cudaError_t dispatch(int64_t items, int r, int64_t ld, const float *A, const float *G, int rs,
                     const float *Xin, float *Xout, int sweeps, const HEpilogue &hep,
                     const WEpilogue &wep, cudaStream_t st) {
    const int T = pick_lanes(r);
    const int need = (r + T - 1) / T < 2 ? 2 : (r + T - 1) / T;
#define NMF_HALS_CASE(TV, SV)                                                                \
    case SV:                                                                                 \
        return hals_launch<TV, SV, LAYOUT>(items, r, ld, A, G, rs, Xin, Xout, sweeps, hep, wep, \
                                           cta_threads(items, T), st);
    if (T == 2) {
        switch (pick(kSlots2, need)) {
            NMF_HALS_CASE(2, 2) NMF_HALS_CASE(2, 3) NMF_HALS_CASE(2, 4) NMF_HALS_CASE(2, 5)
            NMF_HALS_CASE(2, 6) NMF_HALS_CASE(2, 7) NMF_HALS_CASE(2, 8) NMF_HALS_CASE(2, 9)
            NMF_HALS_CASE(2, 10) NMF_HALS_CASE(2, 11) NMF_HALS_CASE(2, 12) NMF_HALS_CASE(2, 13)
            NMF_HALS_CASE(2, 14) NMF_HALS_CASE(2, 15) NMF_HALS_CASE(2, 16) NMF_HALS_CASE(2, 17)
            NMF_HALS_CASE(2, 18) NMF_HALS_CASE(2, 19) NMF_HALS_CASE(2, 20) NMF_HALS_CASE(2, 21)
            NMF_HALS_CASE(2, 22) NMF_HALS_CASE(2, 23) NMF_HALS_CASE(2, 24) NMF_HALS_CASE(2, 25)
            NMF_HALS_CASE(2, 26) NMF_HALS_CASE(2, 27) NMF_HALS_CASE(2, 28) NMF_HALS_CASE(2, 29)
            NMF_HALS_CASE(2, 30) NMF_HALS_CASE(2, 31) NMF_HALS_CASE(2, 32)
            default: break;
        }
    } else {
        switch (pick(kSlots4, need)) {
            NMF_HALS_CASE(4, 17) NMF_HALS_CASE(4, 18) NMF_HALS_CASE(4, 19) NMF_HALS_CASE(4, 20)
            NMF_HALS_CASE(4, 21) NMF_HALS_CASE(4, 22) NMF_HALS_CASE(4, 23) NMF_HALS_CASE(4, 24)
            NMF_HALS_CASE(4, 25) NMF_HALS_CASE(4, 26) NMF_HALS_CASE(4, 27) NMF_HALS_CASE(4, 28)
            NMF_HALS_CASE(4, 29) NMF_HALS_CASE(4, 30) NMF_HALS_CASE(4, 31) NMF_HALS_CASE(4, 32)
            default: break;
        }
    }
#undef NMF_HALS_CASE
    return cudaErrorInvalidValue;
}

}  // namespace

int hals_w_num_ctas(int64_t m, int r) {
    const int T = pick_lanes(r);
    const int64_t per_cta = cta_threads(m, T) / T;
    return (int)((m + per_cta - 1) / per_cta);
}

cudaError_t launch_hals_w(int64_t m, int r, int rs, const float *C, const float *D,
                          const float *W_in, float *W_out, int sweeps, const WEpilogue &ep,
                          cudaStream_t st) {
    HEpilogue none{};
    return dispatch<1>(m, r, rs, C, D, rs, W_in, W_out, sweeps, none, ep, st);
}


// ------------------------------------------------------------ grouped launches
// Key: lanes T, slots S and CTA size of the item's single launch, so that a
// grouped item runs the same CTAs (and sums its error partials in the same
// order) as its single launch.
int hals_w_group_key(int64_t m, int r) {
    const int T = pick_lanes(r);
    const int need = (r + T - 1) / T < 2 ? 2 : (r + T - 1) / T;
    const int S = T == 2 ? pick(kSlots2, need) : pick(kSlots4, need);
    if (S < 0) return -1;
    return (T * 100 + S) * 8 + cta_threads(m, T) / 32;
}

void plan_hals_w_item(int64_t m, int r, int rs, const float *C, const float *D,
                      const float *W_in, float *W_out, int sweeps, const WEpilogue &ep,
                      HalsWItem *it, int64_t *ctas) {
    const int64_t nblk = hals_w_num_ctas(m, r);
    *it = HalsWItem{m, r, rs, C, D, rs, W_in, W_out, sweeps, ep, nblk};
    *ctas = nblk;
}

cudaError_t launch_hals_w_grouped(int key, const HalsWItem *items, const int64_t *begin,
                                  int nitems, int64_t ctas, cudaStream_t st) {
    const int threads = (key % 8) * 32, TS = key / 8;
    const int T = TS / 100, S = TS % 100;
#define NMF_HALS_GROUPED(TV, SV)                                                               \
    if (T == TV && S == SV)                                                                    \
        return hals_w_launch_grouped<TV, SV>(items, begin, nitems, ctas, threads, st);
    NMF_HALS_GROUPED(2, 2) NMF_HALS_GROUPED(2, 3) NMF_HALS_GROUPED(2, 4) NMF_HALS_GROUPED(2, 5)
    NMF_HALS_GROUPED(2, 6) NMF_HALS_GROUPED(2, 7) NMF_HALS_GROUPED(2, 8) NMF_HALS_GROUPED(2, 9)
    NMF_HALS_GROUPED(2, 10) NMF_HALS_GROUPED(2, 11) NMF_HALS_GROUPED(2, 12) NMF_HALS_GROUPED(2, 13)
    NMF_HALS_GROUPED(2, 14) NMF_HALS_GROUPED(2, 15) NMF_HALS_GROUPED(2, 16) NMF_HALS_GROUPED(2, 17)
    NMF_HALS_GROUPED(2, 18) NMF_HALS_GROUPED(2, 19) NMF_HALS_GROUPED(2, 20) NMF_HALS_GROUPED(2, 21)
    NMF_HALS_GROUPED(2, 22) NMF_HALS_GROUPED(2, 23) NMF_HALS_GROUPED(2, 24) NMF_HALS_GROUPED(2, 25)
    NMF_HALS_GROUPED(2, 26) NMF_HALS_GROUPED(2, 27) NMF_HALS_GROUPED(2, 28) NMF_HALS_GROUPED(2, 29)
    NMF_HALS_GROUPED(2, 30) NMF_HALS_GROUPED(2, 31) NMF_HALS_GROUPED(2, 32)
    NMF_HALS_GROUPED(4, 17) NMF_HALS_GROUPED(4, 18) NMF_HALS_GROUPED(4, 19) NMF_HALS_GROUPED(4, 20)
    NMF_HALS_GROUPED(4, 21) NMF_HALS_GROUPED(4, 22) NMF_HALS_GROUPED(4, 23) NMF_HALS_GROUPED(4, 24)
    NMF_HALS_GROUPED(4, 25) NMF_HALS_GROUPED(4, 26) NMF_HALS_GROUPED(4, 27) NMF_HALS_GROUPED(4, 28)
    NMF_HALS_GROUPED(4, 29) NMF_HALS_GROUPED(4, 30) NMF_HALS_GROUPED(4, 31) NMF_HALS_GROUPED(4, 32)
#undef NMF_HALS_GROUPED
    return cudaErrorInvalidValue;
}

}  // namespace nmfg
