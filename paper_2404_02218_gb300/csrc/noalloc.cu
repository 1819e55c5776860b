// FP64 reduction of a dense device array that allocates no device memory.
//
// Some callers cannot allocate device memory at the point where they need a
// reduction: applications whose device memory is entirely owned by their own
// pool (so a cudaMalloc from a library would fail or break their accounting),
// and latency-critical loops where cudaMalloc/cudaFree are off limits because
// they can synchronise the whole device.  This entry point serves them: the
// caller passes the input array and a device location for the result, and the
// per-block partial sums go to a fixed-size array that lives in this library's
// own device image (a file-scope __device__ array), not in allocated memory.
#include <mutex>

#include "gbst_internal.h"

namespace gbst {
namespace {

constexpr int kThreads = 256;
constexpr int kItemsPerThread = 256;                    // elements per thread per block chunk
constexpr int64_t kChunk = int64_t(kThreads) * kItemsPerThread;  // elements per block (65536)
constexpr int kMaxPartials = 16384;                      // 128 KB of FP64 partials
constexpr int64_t kMaxElems = kChunk * kMaxPartials;     // 2^30 elements

// The scratch of every call, on every device that loads the library.  Host code
// must not pass this name to a kernel (on the host it is only a stand-in); it
// passes the device address obtained from cudaGetSymbolAddress instead.
static __device__ __align__(256) double g_partials[kMaxPartials];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double *g_partials_addr[kMaxDevices] = {};

__device__ __forceinline__ double load_elem(const void *p, int dtype, int64_t i)
{
    if (dtype == GBST_F64)
        return static_cast<const double *>(p)[i];
    if (dtype == GBST_F32)
        return static_cast<double>(static_cast<const float *>(p)[i]);
    return static_cast<double>(__bfloat162float(static_cast<const __nv_bfloat16 *>(p)[i]));
}

__device__ __forceinline__ double combine(int kind, double a, double b)
{
    return kind == GBST_RED_MAXABS ? fmax(a, b) : a + b;
}

__device__ __forceinline__ double block_reduce(int kind, double v)
{
    __shared__ double sh[kThreads / 32];
    for (int o = 16; o > 0; o >>= 1)
        v = combine(kind, v, __shfl_down_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0)
        sh[threadIdx.x >> 5] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x < 32) {
        r = threadIdx.x < kThreads / 32 ? sh[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1)
            r = combine(kind, r, __shfl_down_sync(0xffffffffu, r, o));
    }
    return r;
}

// Block b reduces elements [b*kChunk, min(n, (b+1)*kChunk)) and writes partials[b].
__global__ void __launch_bounds__(kThreads) k_partials(const void *x, int dtype, int64_t n, int kind,
                                                       double *partials)
{
    const int64_t begin = static_cast<int64_t>(blockIdx.x) * kChunk;
    const int64_t end = begin + kChunk < n ? begin + kChunk : n;
    double acc = 0.0;
    for (int64_t i = begin + threadIdx.x; i < end; i += kThreads) {
        const double v = load_elem(x, dtype, i);
        acc = combine(kind, acc, kind == GBST_RED_SUM ? v : kind == GBST_RED_L2SQ ? v * v : fabs(v));
    }
    const double r = block_reduce(kind, acc);
    if (threadIdx.x == 0)
        partials[blockIdx.x] = r;
}

__global__ void __launch_bounds__(kThreads) k_final(const double *partials, int nparts, int kind, double *out)
{
    double acc = 0.0;
    for (int i = threadIdx.x; i < nparts; i += kThreads)
        acc = combine(kind, acc, partials[i]);
    const double r = block_reduce(kind, acc);
    if (threadIdx.x == 0)
        *out = r;
}

}  // namespace
}  // namespace gbst

using namespace gbst;

extern "C" gbst_status gbst_reduce_dense_f64_noalloc(const void *x, int dtype, int64_t n, int kind, double *out,
                                                     void *stream)
{
    if (!out || (n > 0 && !x))
        return record_error(GBST_EINVAL, "gbst_reduce_dense_f64_noalloc: null input or output");
    if (dtype != GBST_F32 && dtype != GBST_F64 && dtype != GBST_BF16)
        return record_error(GBST_EINVAL, "gbst_reduce_dense_f64_noalloc: dtype must be F32, F64 or BF16");
    if (kind != GBST_RED_SUM && kind != GBST_RED_L2SQ && kind != GBST_RED_MAXABS)
        return record_error(GBST_EINVAL, "gbst_reduce_dense_f64_noalloc: kind must be SUM, L2SQ or MAXABS");
    if (n < 0 || n > kMaxElems)
        return record_error(
            GBST_EINVAL, "gbst_reduce_dense_f64_noalloc: n must be in [0, 2^30] (the fixed scratch holds 16384 "
                         "block partials of 65536 elements each)");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return record_error(GBST_ECUDA, "gbst_reduce_dense_f64_noalloc: no current CUDA device");
    double *partials = nullptr;
    {
        // One-time set-up per device, with that device current: the device
        // address of the scratch array.
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_partials_addr[dev]) {
            void *p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, g_partials);
            if (e != cudaSuccess || !p)
                return record_error(GBST_ECUDA, "gbst_reduce_dense_f64_noalloc: cudaGetSymbolAddress failed");
            g_partials_addr[dev] = static_cast<double *>(p);
        }
        partials = g_partials_addr[dev];
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int nparts = static_cast<int>((n + kChunk - 1) / kChunk);
    if (nparts > 0)
        k_partials<<<nparts, kThreads, 0, s>>>(x, dtype, n, kind, partials);
    k_final<<<1, kThreads, 0, s>>>(partials, nparts, kind, out);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return record_error(GBST_ECUDA, cudaGetErrorString(e));
    return GBST_OK;
}
