// Streaming (2.5D) star-stencil sweep for sm_103a.
//
// One CTA owns an x-y tile and marches along z.  Every z-plane of the input
// field (tile plus an r-wide halo, 16 bytes wide in x) is copied from HBM to
// shared memory by a TMA tensor load (cp.async.bulk.tensor.3d) that completes
// on an mbarrier; a ring of S = r + 1 + D plane slots keeps the planes
// [z-r, z] resident while the next D planes are in flight.  Each thread owns
// PY rows x PX consecutive x points (16 bytes of storage per row) and keeps
// its 2r+1 z-neighbours in a register queue whose slot indices are resolved at
// compile time by unrolling the z-loop by 2r+1.  x- and y-neighbours are read
// from the centre plane in shared memory with 16-byte loads.
//
// Update (paper Section 5.1 heat listing, Section 6.1 acoustic wave):
//   heat:  u+ = u + a * L(u)
//   wave:  u+ = 2u - u- + kappa * L(u)   (written in place over u-)
//   L(u)  = w0*ndim*u + sum_{m=1..r} w_m [(x-m + x+m) + (y-m + y+m) + (z-m + z+m)]
// The summation order per point is fixed and independent of the point's
// position in its tile, so a decomposed run matches an undecomposed one bit
// for bit.
#include "gbst_internal.h"

namespace gbst {
namespace {

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait on an mbarrier phase; false if it did not complete within kWaitLimitNs.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity)
{
    if (mbar_try_wait(bar, parity))
        return true;
    const unsigned long long t0 = global_ns();
    while (!mbar_try_wait(bar, parity)) {
        if (global_ns() - t0 > kWaitLimitNs)
            return false;
    }
    return true;
}

__device__ __forceinline__ void tma_load_plane(void *dst, const CUtensorMap *map, uint64_t *bar, int x, int y,
                                               int z)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ uint4 lds128(const unsigned char *p)
{
    return *reinterpret_cast<const uint4 *>(p);
}

// ---- storage traits: 16 bytes = PX elements --------------------------------
template <int ST>
struct Storage;

template <>
struct Storage<GBST_F32> {
    static constexpr int PX = 4, ES = 4;
    __device__ __forceinline__ static float get(const uint4 &v, int i)
    {
        return __uint_as_float(i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w);
    }
    __device__ __forceinline__ static uint4 pack(const float *o)
    {
        return make_uint4(__float_as_uint(o[0]), __float_as_uint(o[1]), __float_as_uint(o[2]),
                          __float_as_uint(o[3]));
    }
    __device__ __forceinline__ static void store1(void *p, float v) { *reinterpret_cast<float *>(p) = v; }
};

template <>
struct Storage<GBST_BF16> {
    static constexpr int PX = 8, ES = 2;
    __device__ __forceinline__ static float get(const uint4 &v, int i)
    {
        const uint32_t w = (i >> 1) == 0 ? v.x : (i >> 1) == 1 ? v.y : (i >> 1) == 2 ? v.z : v.w;
        return __uint_as_float((i & 1) ? (w & 0xffff0000u) : (w << 16));
    }
    __device__ __forceinline__ static uint32_t pk2(float lo, float hi)
    {
        const uint32_t l = __bfloat16_as_ushort(__float2bfloat16_rn(lo));
        const uint32_t h = __bfloat16_as_ushort(__float2bfloat16_rn(hi));
        return l | (h << 16);
    }
    __device__ __forceinline__ static uint4 pack(const float *o)
    {
        return make_uint4(pk2(o[0], o[1]), pk2(o[2], o[3]), pk2(o[4], o[5]), pk2(o[6], o[7]));
    }
    __device__ __forceinline__ static void store1(void *p, float v)
    {
        *reinterpret_cast<__nv_bfloat16 *>(p) = __float2bfloat16_rn(v);
    }
};

__device__ __forceinline__ float4 ldg_f4_nc(const float *p)
{
    return __ldg(reinterpret_cast<const float4 *>(p));
}

template <int R, int EQ, int ST, bool HAS_Z, int NT, int PY, int D>
__global__ void __launch_bounds__(NT) k_stream(const SweepArgs a, const int slot_bytes)
{
    using St = Storage<ST>;
    constexpr int PX = St::PX;
    constexpr int ES = St::ES;
    constexpr int G = PX;               // x halo in elements (16 bytes)
    constexpr int RZ = HAS_Z ? R : 0;   // z radius
    constexpr int QN = 2 * RZ + 1;      // register queue length
    constexpr int S = RZ + 1 + D;       // plane slots
    constexpr int NB = D + 1;           // mbarriers (= loads in flight)
    static_assert(R <= G, "x halo must cover the radius");

    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem);
    unsigned char *slots = smem + 128;

    const int tid = threadIdx.x;
    if (blockIdx.x >= a.nunits)
        return;

    if (tid == 0) {
#pragma unroll
        for (int b = 0; b < NB; ++b)
            mbar_init(&bars[b], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    // ---- producer cursor (used by thread 0 only) ----
    int p_unit = blockIdx.x, p_l = 0, p_L = 0;
    Unit pu{};
    auto p_load_unit = [&]() {
        if (p_unit < a.nunits) {
            pu = a.units[p_unit];
            p_L = (pu.z1 - pu.z0) + 2 * RZ;
        }
    };
    auto p_issue = [&](int it) {
        const GridDev &g = a.grids[pu.grid];
        const int TX = g.txt * PX;
        const int TY = (NT / g.txt) * PY;
        const int tile_x = pu.tile % g.tiles_x, tile_y = pu.tile / g.tiles_x;
        uint64_t *bar = &bars[it % NB];
        mbar_arrive_expect_tx(bar, static_cast<uint32_t>(g.box_bytes));
        tma_load_plane(slots + (it % S) * slot_bytes, &g.tmap[a.parity], bar, tile_x * TX, tile_y * TY,
                       pu.z0 + p_l);
        if (++p_l == p_L) {
            p_l = 0;
            p_unit += gridDim.x;
            p_load_unit();
        }
    };
    int p_next = 0;  // next iteration index the producer will issue
    if (tid == 0) {
        p_load_unit();
        for (; p_next < NB && p_unit < a.nunits; ++p_next)
            p_issue(p_next);
    }

    float q[QN][PY][PX];  // z-queue of the thread's own points (values of planes by local index mod QN)
    int j = 0;            // consumer iteration (global over this CTA's units)
    bool failed = false;

    for (int ui = blockIdx.x; ui < a.nunits; ui += gridDim.x) {
        const Unit u = a.units[ui];
        const GridDev &g = a.grids[u.grid];
        const int txt = g.txt;
        const int tx = tid % txt, ty = tid / txt;
        const int TX = txt * PX, TY = (NT / txt) * PY;
        const int tile_x = u.tile % g.tiles_x, tile_y = u.tile / g.tiles_x;
        const int x0 = tile_x * TX + tx * PX;
        const int y0 = tile_y * TY + ty * PY;
        const int row_bytes = (TX + 2 * G) * ES;
        const int own_off = (R + ty * PY) * row_bytes + (G + tx * PX) * ES;
        const int L = (u.z1 - u.z0) + 2 * RZ;
        const int64_t nx = g.nx, ny = g.ny;
        const int64_t pitch = g.pitch, rows = g.rows;
        unsigned char *outbase = static_cast<unsigned char *>(g.buf[1 - a.parity]);
        const bool src_unit = (EQ == GBST_WAVE) && g.has_src;
        const float srcv = (EQ == GBST_WAVE && a.srcval) ? a.srcval[u.grid] : 0.0f;

        for (int l0 = 0; l0 < L; l0 += QN) {
#pragma unroll
            for (int k = 0; k < QN; ++k) {
                const int l = l0 + k;
                if (l < L) {
                    const int zc = u.z0 + (l - 2 * RZ);  // interior z of the centre plane
                    const bool has_centre = l >= 2 * RZ;

                    // Wave: kappa and u- of the centre plane, issued before waiting on the TMA.
                    float kap[PY][PX], um[PY][PX];
                    if (EQ == GBST_WAVE && has_centre) {
#pragma unroll
                        for (int r_ = 0; r_ < PY; ++r_) {
                            const int64_t y = y0 + r_;
                            const bool ok = y < ny && x0 < nx;
                            const float *kp = g.kappa + g.korigin + (zc * g.krows + y) * g.kpitch + x0;
                            const unsigned char *up =
                                outbase + (g.origin + (zc * rows + y) * pitch + x0) * ES;
#pragma unroll
                            for (int v = 0; v < PX / 4; ++v) {
                                const float4 kv = ok ? ldg_f4_nc(kp + 4 * v) : make_float4(0, 0, 0, 0);
                                kap[r_][4 * v + 0] = kv.x;
                                kap[r_][4 * v + 1] = kv.y;
                                kap[r_][4 * v + 2] = kv.z;
                                kap[r_][4 * v + 3] = kv.w;
                            }
                            const uint4 uv = ok ? __ldcs(reinterpret_cast<const uint4 *>(up)) : make_uint4(0, 0, 0, 0);
#pragma unroll
                            for (int i = 0; i < PX; ++i)
                                um[r_][i] = St::get(uv, i);
                        }
                    }

                    // Newest plane: wait for its TMA and push the thread's own points.
                    const unsigned char *nb = slots + (j % S) * slot_bytes;
                    const bool ok = !failed && mbar_wait_bounded(&bars[j % NB], (j / NB) & 1);
                    failed = !ok;
                    if (ok) {
#pragma unroll
                        for (int r_ = 0; r_ < PY; ++r_) {
                            const uint4 v = lds128(nb + own_off + r_ * row_bytes);
#pragma unroll
                            for (int i = 0; i < PX; ++i)
                                q[k][r_][i] = St::get(v, i);
                        }
                    }

                    if (ok && has_centre) {
                        const int kc = (k - RZ + QN) % QN;  // queue slot of the centre plane (constant after unrolling)
                        const unsigned char *cb = slots + ((j - RZ) % S) * slot_bytes + own_off;
                        uint4 ylo[R], yhi[R], xl[PY], xr[PY];
#pragma unroll
                        for (int m = 1; m <= R; ++m) {
                            ylo[m - 1] = lds128(cb - m * row_bytes);
                            yhi[m - 1] = lds128(cb + (PY - 1 + m) * row_bytes);
                        }
#pragma unroll
                        for (int r_ = 0; r_ < PY; ++r_) {
                            xl[r_] = lds128(cb + r_ * row_bytes - 16);
                            xr[r_] = lds128(cb + r_ * row_bytes + 16);
                        }

                        float o[PY][PX];
#pragma unroll
                        for (int r_ = 0; r_ < PY; ++r_) {
#pragma unroll
                            for (int i = 0; i < PX; ++i) {
                                const float c = q[kc][r_][i];
                                float s = a.wc * c;
#pragma unroll
                                for (int m = 1; m <= R; ++m) {
                                    // x neighbours
                                    const int il = i - m, ir = i + m;
                                    const float xm = il >= 0 ? q[kc][r_][il < 0 ? 0 : il]
                                                             : St::get(xl[r_], il < 0 ? PX + il : 0);
                                    const float xp = ir < PX ? q[kc][r_][ir < PX ? ir : 0]
                                                             : St::get(xr[r_], ir >= PX ? ir - PX : 0);
                                    // y neighbours
                                    const int rl = r_ - m, rr = r_ + m;
                                    const float ym = rl >= 0 ? q[kc][rl < 0 ? 0 : rl][i]
                                                             : St::get(ylo[rl < 0 ? -rl - 1 : 0], i);
                                    const float yp = rr < PY ? q[kc][rr < PY ? rr : 0][i]
                                                             : St::get(yhi[rr >= PY ? rr - PY : 0], i);
                                    s = fmaf(a.w[m], xm + xp, s);
                                    s = fmaf(a.w[m], ym + yp, s);
                                    if (HAS_Z) {
                                        const float zm = q[(kc - m + 2 * QN) % QN][r_][i];
                                        const float zp = q[(kc + m) % QN][r_][i];
                                        s = fmaf(a.w[m], zm + zp, s);
                                    }
                                }
                                if (EQ == GBST_HEAT)
                                    o[r_][i] = fmaf(a.a, s, c);
                                else
                                    o[r_][i] = fmaf(kap[r_][i], s, fmaf(2.0f, c, -um[r_][i]));
                            }
                        }
                        if (src_unit && zc == g.src_z) {
                            const int sr = g.src_y - y0, si = g.src_x - x0;
                            if (sr >= 0 && sr < PY && si >= 0 && si < PX) {
#pragma unroll
                                for (int r_ = 0; r_ < PY; ++r_)
#pragma unroll
                                    for (int i = 0; i < PX; ++i)
                                        if (r_ == sr && i == si)
                                            o[r_][i] += srcv;
                            }
                        }
#pragma unroll
                        for (int r_ = 0; r_ < PY; ++r_) {
                            const int64_t y = y0 + r_;
                            if (y < ny) {
                                unsigned char *op = outbase + (g.origin + (zc * rows + y) * pitch + x0) * ES;
                                if (x0 + PX <= nx) {
                                    *reinterpret_cast<uint4 *>(op) = St::pack(o[r_]);
                                } else {
#pragma unroll
                                    for (int i = 0; i < PX; ++i)
                                        if (x0 + i < nx)
                                            St::store1(op + i * ES, o[r_][i]);
                                }
                            }
                        }
                    }

                    // All reads of slot (j - RZ) and of barrier j are done: recycle them.
                    if (__syncthreads_or(failed ? 1 : 0)) {
                        if (tid == 0) {
                            atomicExch(a.err, kDevTimeoutTma);
                            // drain the loads still in flight (bounded) before leaving
                            for (int it = j; it < p_next; ++it)
                                (void)mbar_wait_bounded(&bars[it % NB], (it / NB) & 1);
                        }
                        return;
                    }
                    if (tid == 0 && p_unit < a.nunits) {
                        p_issue(p_next);
                        ++p_next;
                    }
                    ++j;
                }
            }
        }
    }
}

// ---- variant table ---------------------------------------------------------
using KernelFn = void (*)(const SweepArgs, const int);

template <int R, int EQ, int ST, bool HZ, int NT, int PY, int D>
constexpr KernelFn kfn()
{
    return &k_stream<R, EQ, ST, HZ, NT, PY, D>;
}

struct Entry {
    StreamVariant v;
    KernelFn fn;
};

#define GBST_V(R, EQ, ST, HZ, NT, PY, D) \
    Entry{StreamVariant{R, EQ, ST, HZ, NT, PY, D}, kfn<R, EQ, ST, HZ, NT, PY, D>()}

#define GBST_V_EQ_ST(R, HZ, NT, PYF, PYB, D)                                                             \
    GBST_V(R, GBST_HEAT, GBST_F32, HZ, NT, PYF, D), GBST_V(R, GBST_WAVE, GBST_F32, HZ, NT, PYF, D),     \
        GBST_V(R, GBST_HEAT, GBST_BF16, HZ, NT, PYB, D), GBST_V(R, GBST_WAVE, GBST_BF16, HZ, NT, PYB, D)

#define GBST_V_R(HZ, NT, PYF, PYB, D) \
    GBST_V_EQ_ST(1, HZ, NT, PYF, PYB, D), GBST_V_EQ_ST(2, HZ, NT, PYF, PYB, D), GBST_V_EQ_ST(4, HZ, NT, PYF, PYB, D)

const Entry kTable[] = {
    GBST_V_R(true, 128, 2, 1, 3),
    GBST_V_R(false, 128, 2, 1, 3),
};

const Entry *find(const StreamVariant &v)
{
    for (const Entry &e : kTable)
        if (e.v.R == v.R && e.v.eq == v.eq && e.v.storage == v.storage && e.v.has_z == v.has_z &&
            e.v.nthreads == v.nthreads && e.v.py == v.py && e.v.depth == v.depth)
            return &e;
    return nullptr;
}

}  // namespace

bool stream_variant_exists(const StreamVariant &v) { return find(v) != nullptr; }

size_t stream_smem_bytes(const StreamVariant &v, int max_box_bytes)
{
    const int rz = v.has_z ? v.R : 0;
    const int slots = rz + 1 + v.depth;
    const size_t slot = (static_cast<size_t>(max_box_bytes) + 127) / 128 * 128;
    return 128 + slots * slot;
}

// Allow the kernel the device's whole opt-in shared memory once, so handles with
// different slot sizes can share the function.
static bool allow_max_smem(const Entry *e)
{
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
        return false;
    return cudaFuncSetAttribute(reinterpret_cast<const void *>(e->fn), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                optin) == cudaSuccess;
}

int stream_occupancy(const StreamVariant &v, size_t smem)
{
    const Entry *e = find(v);
    if (!e)
        return 0;
    if (!allow_max_smem(e))
        return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, e->fn, v.nthreads, smem) != cudaSuccess)
        return 0;
    return n;
}

cudaError_t launch_stream_sweep(const StreamVariant &v, const SweepArgs &a, int ctas, size_t smem,
                                cudaStream_t s)
{
    const Entry *e = find(v);
    if (!e)
        return cudaErrorInvalidDeviceFunction;
    const int rz = v.has_z ? v.R : 0;
    const int slots = rz + 1 + v.depth;
    const int slot_bytes = static_cast<int>((smem - 128) / slots);
    e->fn<<<ctas, v.nthreads, smem, s>>>(a, slot_bytes);
    return cudaGetLastError();
}

}  // namespace gbst
