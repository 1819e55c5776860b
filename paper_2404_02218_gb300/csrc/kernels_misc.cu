// Supporting kernels: the one-thread-per-point sweep, halo copies (dmp.swap
// faces and periodic wrap), dense <-> padded field transfers and the FP64
// reductions.
#include <algorithm>

#include "gbst_internal.h"

namespace gbst {
namespace {

template <int ST>
struct Elem;
template <>
struct Elem<GBST_F32> {
    using T = float;
    __device__ __forceinline__ static float ld(const T *p) { return *p; }
    __device__ __forceinline__ static void st(T *p, float v) { *p = v; }
};
template <>
struct Elem<GBST_BF16> {
    using T = __nv_bfloat16;
    __device__ __forceinline__ static float ld(const T *p) { return __bfloat162float(*p); }
    __device__ __forceinline__ static void st(T *p, float v) { *p = __float2bfloat16_rn(v); }
};

// ---------------------------------------------------------------------------
// One thread per interior point.  Same per-point arithmetic (and order) as the
// streaming kernel, so both give bit-identical results.
template <int R, int EQ, int ST>
__global__ void k_simple(const SweepArgs a)
{
    using E = Elem<ST>;
    using T = typename E::T;
    const GridDev &g = a.grids[blockIdx.y];
    const int64_t nx = g.nx, ny = g.ny, nz = g.nz;
    const int64_t n = nx * ny * nz;
    const int64_t sy = g.pitch, sz = g.pitch * g.rows;
    const T *u = static_cast<const T *>(g.buf[a.parity]) + g.origin;
    T *out = static_cast<T *>(g.buf[1 - a.parity]) + g.origin;
    const bool has_z = a.ndim == 3;
    for (int64_t p = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; p < n;
         p += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t x = p % nx, y = (p / nx) % ny, z = p / (nx * ny);
        const int64_t idx = z * sz + y * sy + x;
        const float c = E::ld(u + idx);
        float s = a.wc * c;
#pragma unroll
        for (int m = 1; m <= R; ++m) {
            const float xm = E::ld(u + idx - m), xp = E::ld(u + idx + m);
            const float ym = E::ld(u + idx - m * sy), yp = E::ld(u + idx + m * sy);
            float t = (xm + xp) + (ym + yp);
            if (has_z) {
                const float zm = E::ld(u + idx - m * sz), zp = E::ld(u + idx + m * sz);
                t = t + (zm + zp);
            }
            s = fmaf(a.w[m], t, s);
        }
        float o;
        if (EQ == GBST_HEAT) {
            o = fmaf(g.heat_a, s, c);
        } else {
            const float kap = g.kappa[g.korigin + z * g.kpitch * g.krows + y * g.kpitch + x];
            const float um = E::ld(out + idx);
            o = fmaf(kap, __fmul_rn(s, a.lscale), (c + c) - um);
            if (g.has_src && a.srcval && x == g.src_x && y == g.src_y && z == g.src_z)
                o += a.srcval[blockIdx.y];
        }
        E::st(out + idx, o);
    }
}

using SimpleFn = void (*)(const SweepArgs);
template <int EQ, int ST>
SimpleFn simple_for_r(int R)
{
    switch (R) {
    case 1: return &k_simple<1, EQ, ST>;
    case 2: return &k_simple<2, EQ, ST>;
    case 4: return &k_simple<4, EQ, ST>;
    default: return nullptr;
    }
}

// ---------------------------------------------------------------------------
// dmp.swap face copies.  One 1D launch covers every box: box b owns blocks
// [blk0, blk0 + nblk) (found by binary search over blk0).  Rows of ex elements:
// boxes with long rows (faces normal to y or z) give each warp one row at a
// time, moved in 16-byte pieces when the row's two ends allow it; boxes with
// short rows (faces normal to x) give each thread one 16-byte piece when rows
// and starts allow it, else one element.  Index
// arithmetic is 32-bit (a box holds fewer than 2^31 elements; checked on the host).
constexpr int kCopyThreads = 256;
constexpr int kCopyLongRow = 32;  // rows of at least this many elements go warp-per-row

__global__ void __launch_bounds__(kCopyThreads) k_halo_copies(const GridDev *grids, const CopyBox *boxes, int nboxes,
                                                              int parity, int es)
{
    int lo = 0, hi = nboxes - 1;
    const int blk = static_cast<int>(blockIdx.x);
    while (lo < hi) {  // last box with blk0 <= blk
        const int mid = (lo + hi + 1) >> 1;
        if (boxes[mid].blk0 <= blk)
            lo = mid;
        else
            hi = mid - 1;
    }
    const CopyBox b = boxes[lo];
    const uint32_t bb = static_cast<uint32_t>(blk - b.blk0), nb = static_cast<uint32_t>(b.nblk);
    const GridDev &gs = grids[b.src_grid];
    const GridDev &gd = grids[b.dst_grid];
    const unsigned char *src = static_cast<const unsigned char *>(gs.buf[parity]) + b.src_off;
    unsigned char *dst = static_cast<unsigned char *>(gd.buf[parity]) + b.dst_off;
    const uint32_t ex = static_cast<uint32_t>(b.ex), ey = static_cast<uint32_t>(b.ey);
    const uint32_t nrows = ey * static_cast<uint32_t>(b.ez);
    const int64_t sps = gs.pitch * es, spp = gs.pitch * gs.rows * es;
    const int64_t dps = gd.pitch * es, dpp = gd.pitch * gd.rows * es;
    const uint32_t row_bytes = ex * static_cast<uint32_t>(es);
    if (ex >= kCopyLongRow) {
        const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = kCopyThreads / 32;
        // row starts differ by multiples of the pitch (a multiple of 128 bytes)
        const bool vec = ((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst) | row_bytes) & 15) == 0;
        for (uint32_t row = bb * nw + warp; row < nrows; row += nb * nw) {
            const uint32_t j = row % ey, k = row / ey;
            const unsigned char *s = src + k * spp + j * sps;
            unsigned char *d = dst + k * dpp + j * dps;
            if (vec) {
                for (uint32_t c = lane; c < row_bytes / 16; c += 32)
                    reinterpret_cast<uint4 *>(d)[c] = reinterpret_cast<const uint4 *>(s)[c];
            } else if (es == 4) {
                for (uint32_t i = lane; i < ex; i += 32)
                    reinterpret_cast<uint32_t *>(d)[i] = reinterpret_cast<const uint32_t *>(s)[i];
            } else {
                for (uint32_t i = lane; i < ex; i += 32)
                    reinterpret_cast<uint16_t *>(d)[i] = reinterpret_cast<const uint16_t *>(s)[i];
            }
        }
        return;
    }
    // short rows of whole 16-byte pieces at 16-byte aligned starts (x faces widened to a
    // 32-byte sector): consecutive threads take consecutive pieces of consecutive rows
    if ((row_bytes & 15) == 0 &&
        ((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst) | static_cast<uintptr_t>(sps) |
          static_cast<uintptr_t>(spp) | static_cast<uintptr_t>(dps) | static_cast<uintptr_t>(dpp)) & 15) == 0) {
        const uint32_t cpr = row_bytes >> 4, n = nrows * cpr;
        for (uint32_t t = bb * kCopyThreads + threadIdx.x; t < n; t += nb * kCopyThreads) {
            const uint32_t row = t / cpr, c = t - row * cpr;
            const uint32_t j = row % ey, k = row / ey;
            *reinterpret_cast<uint4 *>(dst + k * dpp + j * dps + c * 16u) =
                *reinterpret_cast<const uint4 *>(src + k * spp + j * sps + c * 16u);
        }
        return;
    }
    // short rows: consecutive threads take consecutive elements of consecutive rows, so a
    // warp's loads and stores cover whole rows' bytes (32 / ex rows per instruction)
    const uint32_t n = nrows * ex;
    for (uint32_t t = bb * kCopyThreads + threadIdx.x; t < n; t += nb * kCopyThreads) {
        const uint32_t row = t / ex, i = t - row * ex;
        const uint32_t j = row % ey, k = row / ey;
        const int64_t so = k * spp + j * sps + static_cast<int64_t>(i) * es;
        const int64_t d = k * dpp + j * dps + static_cast<int64_t>(i) * es;
        if (es == 4)
            *reinterpret_cast<uint32_t *>(dst + d) = *reinterpret_cast<const uint32_t *>(src + so);
        else
            *reinterpret_cast<uint16_t *>(dst + d) = *reinterpret_cast<const uint16_t *>(src + so);
    }
}

// ---------------------------------------------------------------------------
__device__ __forceinline__ double load_dense(const void *p, int dtype, int64_t i)
{
    if (dtype == GBST_F64)
        return static_cast<const double *>(p)[i];
    if (dtype == GBST_F32)
        return static_cast<double>(static_cast<const float *>(p)[i]);
    return static_cast<double>(__bfloat162float(static_cast<const __nv_bfloat16 *>(p)[i]));
}

// FP32 on both sides, rows of a multiple of 4 elements at 16-byte aligned starts:
// a warp per row, 16-byte pieces (a thread per element and a row per block moved
// 1.9 TB/s at 256^3).
__device__ __forceinline__ bool xfer_vec4(const XferArgs &x)
{
    return x.storage == GBST_F32 && x.dense_dtype == GBST_F32 && ((x.nx | x.gx | x.gnx) & 3) == 0 &&
           ((reinterpret_cast<uintptr_t>(x.padded) | reinterpret_cast<uintptr_t>(x.dense)) & 15) == 0 &&
           ((x.origin | x.pitch) & 3) == 0;
}

template <int MODE>  // 0: dense -> padded, 1: padded -> dense, 2: padded += dense
__device__ __forceinline__ void xfer_rows_vec4(const XferArgs &x)
{
    const int64_t nrows = x.ny * x.nz, nx4 = x.nx >> 2;
    const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int64_t row = static_cast<int64_t>(blockIdx.x) * nw + (threadIdx.x >> 5); row < nrows;
         row += static_cast<int64_t>(gridDim.x) * nw) {
        const int64_t j = row % x.ny, k = row / x.ny;
        float4 *pd = reinterpret_cast<float4 *>(static_cast<float *>(x.padded) + x.origin + (k * x.rows + j) * x.pitch);
        float4 *dd = reinterpret_cast<float4 *>(static_cast<float *>(x.dense) +
                                                ((x.gz + k) * x.gny + (x.gy + j)) * x.gnx + x.gx);
        for (int64_t i = lane; i < nx4; i += 32) {
            if (MODE == 0) {
                pd[i] = dd[i];
            } else if (MODE == 1) {
                dd[i] = pd[i];
            } else {
                float4 a = pd[i];
                const float4 b = dd[i];
                a.x += b.x;
                a.y += b.y;
                a.z += b.z;
                a.w += b.w;
                pd[i] = a;
            }
        }
    }
}

// Dense <-> padded transfers, one block per x row (grid-stride over the ny*nz
// rows; one division per row), threads along x: both sides are read and
// written in contiguous runs, which also suits host memory accessed over the
// host link.
__global__ void k_scatter(const XferArgs x)
{
    if (xfer_vec4(x) && !(x.scale_sq > 0.0)) {
        xfer_rows_vec4<0>(x);
        return;
    }
    const int64_t nrows = x.ny * x.nz;
    for (int64_t row = blockIdx.x; row < nrows; row += gridDim.x) {
        const int64_t j = row % x.ny, k = row / x.ny;
        const int64_t d0 = ((x.gz + k) * x.gny + (x.gy + j)) * x.gnx + x.gx;
        const int64_t o0 = x.origin + (k * x.rows + j) * x.pitch;
        if (x.storage == GBST_F32 && x.dense_dtype == GBST_F32 && !(x.scale_sq > 0.0)) {
            const float *src = static_cast<const float *>(x.dense) + d0;
            float *dst = static_cast<float *>(x.padded) + o0;
            for (int64_t i = threadIdx.x; i < x.nx; i += blockDim.x)
                dst[i] = src[i];
            continue;
        }
        for (int64_t i = threadIdx.x; i < x.nx; i += blockDim.x) {
            double v = load_dense(x.dense, x.dense_dtype, d0 + i);
            if (x.scale_sq > 0.0)
                v = v * v * x.scale_sq;
            if (x.storage == GBST_BF16)
                static_cast<__nv_bfloat16 *>(x.padded)[o0 + i] = __double2bfloat16(v);
            else
                static_cast<float *>(x.padded)[o0 + i] = __double2float_rn(v);
        }
    }
}

__global__ void k_gather(const XferArgs x)
{
    if (xfer_vec4(x)) {
        xfer_rows_vec4<1>(x);
        return;
    }
    const int64_t nrows = x.ny * x.nz;
    for (int64_t row = blockIdx.x; row < nrows; row += gridDim.x) {
        const int64_t j = row % x.ny, k = row / x.ny;
        const int64_t d0 = ((x.gz + k) * x.gny + (x.gy + j)) * x.gnx + x.gx;
        const int64_t o0 = x.origin + (k * x.rows + j) * x.pitch;
        for (int64_t i = threadIdx.x; i < x.nx; i += blockDim.x) {
            float v;
            if (x.storage == GBST_BF16)
                v = __bfloat162float(static_cast<const __nv_bfloat16 *>(x.padded)[o0 + i]);
            else
                v = static_cast<const float *>(x.padded)[o0 + i];
            if (x.dense_dtype == GBST_F64)
                static_cast<double *>(x.dense)[d0 + i] = static_cast<double>(v);
            else if (x.dense_dtype == GBST_F32)
                static_cast<float *>(x.dense)[d0 + i] = v;
            else
                static_cast<__nv_bfloat16 *>(x.dense)[d0 + i] = __float2bfloat16_rn(v);
        }
    }
}

__global__ void k_scatter_add(const XferArgs x)
{
    if (xfer_vec4(x)) {
        xfer_rows_vec4<2>(x);
        return;
    }
    const int64_t n = x.nx * x.ny * x.nz;
    for (int64_t p = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; p < n;
         p += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t i = p % x.nx, j = (p / x.nx) % x.ny, k = p / (x.nx * x.ny);
        const int64_t o = x.origin + (k * x.rows + j) * x.pitch + i;
        const float v = static_cast<const float *>(x.dense)[p];
        if (x.storage == GBST_BF16) {
            __nv_bfloat16 *q = static_cast<__nv_bfloat16 *>(x.padded) + o;
            *q = __float2bfloat16_rn(__bfloat162float(*q) + v);
        } else {
            static_cast<float *>(x.padded)[o] += v;
        }
    }
}

__global__ void k_gather_strided(const XferArgs x, int st)
{
    const int64_t mx = (x.nx + st - 1) / st, my = (x.ny + st - 1) / st, mz = (x.nz + st - 1) / st;
    const int64_t n = mx * my * mz;
    for (int64_t p = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; p < n;
         p += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t i = (p % mx) * st, j = ((p / mx) % my) * st, k = (p / (mx * my)) * st;
        const int64_t o = x.origin + (k * x.rows + j) * x.pitch + i;
        static_cast<float *>(x.dense)[p] = x.storage == GBST_BF16
                                               ? __bfloat162float(static_cast<const __nv_bfloat16 *>(x.padded)[o])
                                               : static_cast<const float *>(x.padded)[o];
    }
}

__global__ void k_kappa_to_cnorm(const XferArgs x, double factor)
{
    const int64_t n = x.nx * x.ny * x.nz;
    for (int64_t p = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; p < n;
         p += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t i = p % x.nx, j = (p / x.nx) % x.ny, k = p / (x.nx * x.ny);
        const int64_t o = x.origin + (k * x.rows + j) * x.pitch + i;
        const double kap = static_cast<const float *>(x.padded)[o];
        static_cast<float *>(x.dense)[p] = static_cast<float>(sqrt(kap) * factor);
    }
}

// ---------------------------------------------------------------------------
constexpr int kRedThreads = 256;

__device__ __forceinline__ double combine(int kind, double a, double b)
{
    return kind == GBST_RED_MAXABS ? fmax(a, b) : a + b;
}

template <int ST>
__device__ __forceinline__ double ldd(const void *base, int64_t i)
{
    return static_cast<double>(Elem<ST>::ld(static_cast<const typename Elem<ST>::T *>(base) + i));
}

struct RedW {
    double w[kMaxRadius + 1];
};

template <int ST>
__global__ void __launch_bounds__(kRedThreads) k_reduce(int kind, int ndim, int R, RedW rw,
                                                        const ReduceGrid *grids, int ngrids,
                                                        double *partials)
{
    double acc = 0.0;
    const int bpg = gridDim.x / ngrids;  // blocks per grid
    const int gi = blockIdx.x / bpg;
    const int bi = blockIdx.x % bpg;
    if (gi < ngrids) {
        const ReduceGrid g = grids[gi];
        const int64_t n = g.nx * g.ny * g.nz;
        const int64_t sy = g.pitch, sz = g.pitch * g.rows;
        for (int64_t p = bi * static_cast<int64_t>(blockDim.x) + threadIdx.x; p < n;
             p += static_cast<int64_t>(bpg) * blockDim.x) {
            const int64_t x = p % g.nx, y = (p / g.nx) % g.ny, z = p / (g.nx * g.ny);
            const int64_t idx = g.origin + z * sz + y * sy + x;
            const double u = ldd<ST>(g.u, idx);
            double t;
            if (kind == GBST_RED_SUM) {
                t = u;
            } else if (kind == GBST_RED_L2SQ) {
                t = u * u;
            } else if (kind == GBST_RED_MAXABS) {
                t = fabs(u);
            } else {
                const double v = ldd<ST>(g.v, idx);
                const double kap =
                    static_cast<double>(g.kappa[g.korigin + z * g.kpitch * g.krows + y * g.kpitch + x]);
                double lv = static_cast<double>(ndim) * rw.w[0] * v;
                for (int m = 1; m <= R; ++m) {
                    lv += rw.w[m] * (ldd<ST>(g.v, idx - m) + ldd<ST>(g.v, idx + m));
                    lv += rw.w[m] * (ldd<ST>(g.v, idx - m * sy) + ldd<ST>(g.v, idx + m * sy));
                    if (ndim == 3)
                        lv += rw.w[m] * (ldd<ST>(g.v, idx - m * sz) + ldd<ST>(g.v, idx + m * sz));
                }
                const double d = u - v;
                t = d * d / kap - u * lv;
            }
            acc = combine(kind, acc, t);
        }
    }
    // block reduction in a fixed order
    __shared__ double sh[kRedThreads / 32];
    for (int o = 16; o > 0; o >>= 1)
        acc = combine(kind, acc, __shfl_down_sync(0xffffffffu, acc, o));
    if ((threadIdx.x & 31) == 0)
        sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < kRedThreads / 32 ? sh[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1)
            v = combine(kind, v, __shfl_down_sync(0xffffffffu, v, o));
        if (threadIdx.x == 0)
            partials[blockIdx.x] = v;
    }
}

__global__ void __launch_bounds__(kRedThreads) k_reduce_final(int kind, const double *partials, int n,
                                                              double *out)
{
    double acc = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x)
        acc = combine(kind, acc, partials[i]);
    __shared__ double sh[kRedThreads / 32];
    for (int o = 16; o > 0; o >>= 1)
        acc = combine(kind, acc, __shfl_down_sync(0xffffffffu, acc, o));
    if ((threadIdx.x & 31) == 0)
        sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < kRedThreads / 32 ? sh[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1)
            v = combine(kind, v, __shfl_down_sync(0xffffffffu, v, o));
        if (threadIdx.x == 0)
            *out = v;
    }
}

int grid_for(int64_t n, int threads, int cap)
{
    const int64_t b = (n + threads - 1) / threads;
    return static_cast<int>(b < 1 ? 1 : (b > cap ? cap : b));
}

}  // namespace

cudaError_t launch_simple_sweep(int R, int eq, int storage, const SweepArgs &a, int ngrids, int64_t max_points,
                                cudaStream_t s)
{
    SimpleFn fn = nullptr;
    if (eq == GBST_HEAT)
        fn = storage == GBST_BF16 ? simple_for_r<GBST_HEAT, GBST_BF16>(R) : simple_for_r<GBST_HEAT, GBST_F32>(R);
    else
        fn = storage == GBST_BF16 ? simple_for_r<GBST_WAVE, GBST_BF16>(R) : simple_for_r<GBST_WAVE, GBST_F32>(R);
    if (!fn)
        return cudaErrorInvalidValue;
    dim3 grid(grid_for(max_points, 256, 4096), ngrids);
    fn<<<grid, 256, 0, s>>>(a);
    return cudaGetLastError();
}

int halo_copy_blocks(CopyBox *boxes, int nboxes)
{
    // one row per warp (long rows) or per thread (short rows), at most 2048 blocks per box
    int total = 0;
    for (int i = 0; i < nboxes; ++i) {
        CopyBox &b = boxes[i];
        // long rows: one per warp; short rows: one element per thread
        const int64_t work = b.ex >= kCopyLongRow ? b.ey * b.ez : b.ex * b.ey * b.ez;
        const int64_t per_block = b.ex >= kCopyLongRow ? kCopyThreads / 32 : kCopyThreads;
        b.nblk = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(2048, (work + per_block - 1) / per_block)));
        b.blk0 = total;
        total += b.nblk;
    }
    return total;
}

cudaError_t launch_halo_copies(const GridDev *grids, const CopyBox *boxes, int nboxes, int parity, int elem_size,
                               int total_blocks, cudaStream_t s)
{
    if (nboxes == 0 || total_blocks <= 0)
        return cudaSuccess;
    k_halo_copies<<<total_blocks, kCopyThreads, 0, s>>>(grids, boxes, nboxes, parity, elem_size);
    return cudaGetLastError();
}

cudaError_t launch_scatter(const XferArgs &x, cudaStream_t s)
{
    k_scatter<<<static_cast<unsigned>(std::min<int64_t>(x.ny * x.nz, 16384)), 256, 0, s>>>(x);
    return cudaGetLastError();
}

cudaError_t launch_gather(const XferArgs &x, cudaStream_t s)
{
    k_gather<<<static_cast<unsigned>(std::min<int64_t>(x.ny * x.nz, 16384)), 256, 0, s>>>(x);
    return cudaGetLastError();
}

cudaError_t launch_scatter_add(const XferArgs &x, cudaStream_t s)
{
    k_scatter_add<<<grid_for(x.nx * x.ny * x.nz, 256, 8192), 256, 0, s>>>(x);
    return cudaGetLastError();
}

cudaError_t launch_gather_strided(const XferArgs &x, int stride, cudaStream_t s)
{
    const int64_t n = ((x.nx + stride - 1) / stride) * ((x.ny + stride - 1) / stride) * ((x.nz + stride - 1) / stride);
    k_gather_strided<<<grid_for(n, 256, 8192), 256, 0, s>>>(x, stride);
    return cudaGetLastError();
}

cudaError_t launch_kappa_to_cnorm(const XferArgs &x, double factor, cudaStream_t s)
{
    k_kappa_to_cnorm<<<grid_for(x.nx * x.ny * x.nz, 256, 8192), 256, 0, s>>>(x, factor);
    return cudaGetLastError();
}

int reduce_blocks_for(int64_t points) { return grid_for(points, kRedThreads, 1024); }

cudaError_t launch_reduce_partials(int kind, int storage, int ndim, int R, const double *w,
                                   const ReduceGrid *grids_dev, int ngrids, int64_t max_points, double *partials,
                                   int nblocks, cudaStream_t s)
{
    RedW rw{};
    for (int m = 0; m <= R && m <= kMaxRadius; ++m)
        rw.w[m] = w[m];
    (void)max_points;
    if (storage == GBST_BF16)
        k_reduce<GBST_BF16><<<nblocks, kRedThreads, 0, s>>>(kind, ndim, R, rw, grids_dev, ngrids, partials);
    else
        k_reduce<GBST_F32><<<nblocks, kRedThreads, 0, s>>>(kind, ndim, R, rw, grids_dev, ngrids, partials);
    return cudaGetLastError();
}

cudaError_t launch_reduce_final(int kind, const double *partials, int n, double *out, cudaStream_t s)
{
    k_reduce_final<<<1, kRedThreads, 0, s>>>(kind, partials, n, out);
    return cudaGetLastError();
}

}  // namespace gbst
