// noalloc.cu -- nmf_fro2_noalloc: ||X||_F^2 of a device matrix without any
// device allocation.
//
// Why: some callers cannot call cudaMalloc at the point where they need the
// value -- e.g. code that runs inside another framework's memory budget (the
// framework owns every byte of device memory), or a latency-critical loop in
// which an allocation could block on device-wide synchronisation.  They pass
// their input and output buffers; the reduction's per-CTA partial sums live
// in the fixed array below instead of in allocated scratch.
//
// The scratch is one file-scope __device__ array shared by every call on a
// device (each GPU that loads the library holds it until the process exits).
// Consequences for callers:
//  * calls whose kernels overlap on the GPU (different streams, or host
//    threads without ordering) race on the array -- serialise them;
//  * the array keeps the last call's partial sums; nothing in it has to
//    start at zero, because every call writes each partial it later reads;
//  * host code cannot use the array's name as a device address, so the
//    first call on each device looks the address up with
//    cudaGetSymbolAddress (with that device current) and caches it; make
//    that first call before any stream capture.  The cached address belongs
//    to the device's current context: after a cudaDeviceReset in the same
//    process it is stale, so the entry point must not be used after one.
#include <cuda_runtime.h>

#include <mutex>

#include "common.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int64_t kPerThread = 64;                   // elements summed by one thread
constexpr int kMaxParts = 16384;                     // 16384 FP64 partials = 128 KiB
constexpr int64_t kMaxCount = (int64_t)kMaxParts * kThreads * kPerThread;   // 2^28 entries
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_fro2_scratch[kMaxParts];

std::mutex g_mu;
double *g_scratch_ptr[kMaxDevices] = {};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ double block_sum(double v) {
    __shared__ double red[kThreads / 32];
    v = warp_sum(v);
    if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < kThreads / 32; ++i) s += red[i];
    return s;
}

// CTA b sums the squares of entries [b*256*64, (b+1)*256*64) of the m x n
// matrix (row stride ld) into part[b].
__global__ void __launch_bounds__(kThreads)
fro2_partial_noalloc(const float *__restrict__ X, int64_t n, int64_t ld, int64_t count,
                     double *__restrict__ part) {
    const int64_t base = (int64_t)blockIdx.x * kThreads * kPerThread;
    double acc = 0.0;
    // Entry q = base + u * kThreads + t sits at row q / n, column q % n; the
    // position is divided out once per thread and then advanced by kThreads
    // entries, dividing again only when it wraps into a later row.
    int64_t q = base + threadIdx.x;
    int64_t row = q / n, col = q - row * n;
    for (int64_t u = 0; u < kPerThread && q < count; ++u) {
        const double x = (double)X[row * ld + col];
        acc = fma(x, x, acc);
        q += kThreads;
        col += kThreads;
        if (col >= n) {                          // wrapped into a later row
            const int64_t d = col / n;
            row += d;
            col -= d * n;
        }
    }
    const double s = block_sum(acc);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// One CTA adds the partials in a fixed order.
__global__ void __launch_bounds__(kThreads)
fro2_sum_noalloc(const double *__restrict__ part, int parts, double *__restrict__ out) {
    double acc = 0.0;
    for (int i = threadIdx.x; i < parts; i += kThreads) acc += part[i];
    const double s = block_sum(acc);
    if (threadIdx.x == 0) *out = s;
}

}  // namespace

extern "C" nmf_status nmf_fro2_noalloc(const float *X, int64_t m, int64_t n, int64_t ld,
                                       double *out, void *stream) {
    if (!X || !out) return nmfg::set_error(NMF_EINVAL, "nmf_fro2_noalloc: X and out are required");
    if (m < 1 || n < 1 || ld < n)
        return nmfg::set_error(NMF_EINVAL, "nmf_fro2_noalloc: need m, n >= 1 and ld >= n");
    // Compare before multiplying: m * n itself could overflow int64.
    if (n > kMaxCount / m)
        return nmfg::set_error(NMF_ENOTSUP,
                               "nmf_fro2_noalloc: m*n exceeds 2^28 entries, the capacity of its "
                               "fixed 128 KiB scratch");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return nmfg::set_error(NMF_ECUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices)
        return nmfg::set_error(NMF_ENOTSUP, "nmf_fro2_noalloc: device ordinal out of range");
    double *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        if (!g_scratch_ptr[dev]) {
            // The current device is `dev`, so this resolves its copy of the array.
            e = cudaGetSymbolAddress((void **)&scratch, g_fro2_scratch);
            if (e != cudaSuccess) return nmfg::set_error(NMF_ECUDA, cudaGetErrorString(e));
            g_scratch_ptr[dev] = scratch;
        }
        scratch = g_scratch_ptr[dev];
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int64_t count = m * n;
    const int parts = (int)((count + kThreads * kPerThread - 1) / (kThreads * kPerThread));
    fro2_partial_noalloc<<<parts, kThreads, 0, st>>>(X, n, ld, count, scratch);
    e = cudaGetLastError();
    if (e == cudaSuccess) {
        fro2_sum_noalloc<<<1, kThreads, 0, st>>>(scratch, parts, out);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return nmfg::set_error(NMF_ECUDA, cudaGetErrorString(e));
    return NMF_OK;
}
