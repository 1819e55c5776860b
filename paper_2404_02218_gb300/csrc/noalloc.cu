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
#include <cuda.h>

#include <cstdio>
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

// Device address of g_partials per CUDA context.  The address belongs to one
// context's load of this module, so the cache is keyed on the context's
// process-unique id (cuCtxGetId): a context created after cudaDeviceReset, or a
// non-primary context made current by the caller, gets its own look-up.
constexpr int kMaxContexts = 64;
struct ScratchAddr {
    unsigned long long ctx_id;
    double *addr;
};
std::mutex g_mu;
ScratchAddr g_addr[kMaxContexts] = {};
int g_naddr = 0;

typedef CUresult (*PfnCtxGetCurrent)(CUcontext *);
typedef CUresult (*PfnCtxGetId)(CUcontext, unsigned long long *);

// Id of the calling thread's current context (created by the runtime if none is current yet).
bool current_context_id(unsigned long long *id)
{
    static PfnCtxGetCurrent get_current = nullptr;
    static PfnCtxGetId get_id = nullptr;
    if (!get_current || !get_id) {
        void *p = nullptr, *q = nullptr;
        cudaDriverEntryPointQueryResult r1{}, r2{};
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &r1) != cudaSuccess ||
            r1 != cudaDriverEntryPointSuccess || !p ||
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &q, 12000, cudaEnableDefault, &r2) != cudaSuccess ||
            r2 != cudaDriverEntryPointSuccess || !q) {
            cudaGetLastError();
            return false;
        }
        get_current = reinterpret_cast<PfnCtxGetCurrent>(p);
        get_id = reinterpret_cast<PfnCtxGetId>(q);
    }
    CUcontext ctx = nullptr;
    if (get_current(&ctx) != CUDA_SUCCESS)
        return false;
    if (!ctx) {
        // No context is current on this thread yet: make the current device's
        // primary context current (cudaSetDevice initialises it; nothing is allocated).
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaSetDevice(dev) != cudaSuccess ||
            get_current(&ctx) != CUDA_SUCCESS || !ctx) {
            cudaGetLastError();
            return false;
        }
    }
    return get_id(ctx, id) == CUDA_SUCCESS;
}

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
    static const char *kName = "gbst_reduce_dense_f64_noalloc";
    char msg[256];
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
    unsigned long long ctx_id = 0;
    if (!current_context_id(&ctx_id))
        return record_error(GBST_ECUDA, "gbst_reduce_dense_f64_noalloc: no current CUDA context");
    double *partials = nullptr;
    {
        // One-time set-up per device context, with that context current: the
        // device address of the scratch array.
        std::lock_guard<std::mutex> lk(g_mu);
        for (int i = 0; i < g_naddr; ++i)
            if (g_addr[i].ctx_id == ctx_id)
                partials = g_addr[i].addr;
        if (!partials) {
            void *p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, g_partials);
            if (e != cudaSuccess || !p) {
                snprintf(msg, sizeof msg, "%s: cudaGetSymbolAddress failed (%s)", kName, cudaGetErrorString(e));
                return record_error(GBST_ECUDA, msg);
            }
            partials = static_cast<double *>(p);
            ScratchAddr &slot = g_addr[g_naddr < kMaxContexts ? g_naddr++ : kMaxContexts - 1];
            slot.ctx_id = ctx_id;
            slot.addr = partials;
        }
    }
    // An error left pending by an earlier, unrelated launch would otherwise be
    // reported as this call's failure.
    cudaGetLastError();
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int nparts = static_cast<int>((n + kChunk - 1) / kChunk);
    if (nparts > 0)
        k_partials<<<nparts, kThreads, 0, s>>>(x, dtype, n, kind, partials);
    k_final<<<1, kThreads, 0, s>>>(partials, nparts, kind, out);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        snprintf(msg, sizeof msg, "%s: kernel launch failed (%s)", kName, cudaGetErrorString(e));
        return record_error(GBST_ECUDA, msg);
    }
    return GBST_OK;
}
