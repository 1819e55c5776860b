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
//   L(u)  = w0*ndim*u + sum_{m=1..r} w_m [((x-m + x+m) + (y-m + y+m)) + (z-m + z+m)]
// The weights arrive as integers over a common denominator (exact in FP32, so the
// star of a constant is exactly zero); the heat coefficient a carries the
// denominator, the wave multiplies the sum by its inverse (lscale) before kappa.
// The summation order per point is fixed and independent of the point's
// position in its tile, so a decomposed run matches an undecomposed one bit
// for bit.
#pragma once
#include "gbst_internal.h"

namespace gbst {
namespace sweep {
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
    __device__ __forceinline__ static float2 pair(const uint4 &v, int pp)
    {
        return pp == 0 ? make_float2(__uint_as_float(v.x), __uint_as_float(v.y))
                       : make_float2(__uint_as_float(v.z), __uint_as_float(v.w));
    }
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
    __device__ __forceinline__ static float2 pair(const uint4 &v, int pp)
    {
        const uint32_t w = pp == 0 ? v.x : pp == 1 ? v.y : pp == 2 ? v.z : v.w;
        return make_float2(__uint_as_float(w << 16), __uint_as_float(w & 0xffff0000u));
    }
    __device__ __forceinline__ static float get(const uint4 &v, int i)
    {
        const uint32_t w = (i >> 1) == 0 ? v.x : (i >> 1) == 1 ? v.y : (i >> 1) == 2 ? v.z : v.w;
        return __uint_as_float((i & 1) ? (w & 0xffff0000u) : (w << 16));
    }
    __device__ __forceinline__ static uint32_t pk2(float lo, float hi)
    {
        // both halves rounded to nearest even in one conversion (lo in the low 16 bits)
        const __nv_bfloat162 b = __floats2bfloat162_rn(lo, hi);
        return *reinterpret_cast<const uint32_t *>(&b);
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

// 32-bit word pp of a 16-byte chunk (BF16 storage: the point pair pp)
__device__ __forceinline__ uint32_t word_of(const uint4 &v, int pp)
{
    return pp == 0 ? v.x : pp == 1 ? v.y : pp == 2 ? v.z : v.w;
}

// (lo(a) + lo(b), hi(a) + hi(b)) for two words of BF16 pairs, in FP32 rounded to
// nearest: a's halves are widened, b's halves enter mixed-precision additions.
// Each sum of two BF16 values is the same FP32 value as the packed FP32x2 sum of
// both widened pairs (the operands are exact, the addition commutes).
__device__ __forceinline__ float2 bf16_pair_sum(uint32_t a, uint32_t b)
{
    const float ax = __uint_as_float(a << 16), ay = __uint_as_float(a & 0xffff0000u);
    float2 r;
    asm("{\n\t.reg .b16 l, h;\n\t"
        "mov.b32 {l, h}, %2;\n\t"
        "add.rn.f32.bf16 %0, l, %3;\n\t"
        "add.rn.f32.bf16 %1, h, %4;\n\t}"
        : "=f"(r.x), "=f"(r.y)
        : "r"(b), "f"(ax), "f"(ay));
    return r;
}

// (lo(w) - c.x, hi(w) - c.y) for a word of a BF16 pair, in FP32 rounded to nearest.
__device__ __forceinline__ float2 bf16_pair_sub(uint32_t w, float2 c)
{
    float2 r;
    asm("{\n\t.reg .b16 l, h;\n\t"
        "mov.b32 {l, h}, %2;\n\t"
        "sub.rn.f32.bf16 %0, l, %3;\n\t"
        "sub.rn.f32.bf16 %1, h, %4;\n\t}"
        : "=f"(r.x), "=f"(r.y)
        : "r"(w), "f"(c.x), "f"(c.y));
    return r;
}

// x-halo loads narrowed to the r elements next to the thread's column: the
// returned 16-byte chunk holds them at their natural positions (zero elsewhere).
template <int ST, int R>
__device__ __forceinline__ uint4 load_left(const unsigned char *chunk)
{
    constexpr int B = R * Storage<ST>::ES <= 4 ? 4 : (R * Storage<ST>::ES <= 8 ? 8 : 16);
    uint4 v = make_uint4(0, 0, 0, 0);
    if (B == 4) {
        v.w = *reinterpret_cast<const uint32_t *>(chunk + 12);
    } else if (B == 8) {
        const uint2 t = *reinterpret_cast<const uint2 *>(chunk + 8);
        v.z = t.x;
        v.w = t.y;
    } else {
        v = *reinterpret_cast<const uint4 *>(chunk);
    }
    return v;
}

template <int ST, int R>
__device__ __forceinline__ uint4 load_right(const unsigned char *chunk)
{
    constexpr int B = R * Storage<ST>::ES <= 4 ? 4 : (R * Storage<ST>::ES <= 8 ? 8 : 16);
    uint4 v = make_uint4(0, 0, 0, 0);
    if (B == 4) {
        v.x = *reinterpret_cast<const uint32_t *>(chunk);
    } else if (B == 8) {
        const uint2 t = *reinterpret_cast<const uint2 *>(chunk);
        v.x = t.x;
        v.y = t.y;
    } else {
        v = *reinterpret_cast<const uint4 *>(chunk);
    }
    return v;
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Work-unit source of a streaming launch: unit ui to CTA ui mod gridDim, or,
// with a.dyn, CTA b starts with unit b and then draws gridDim + the next index
// of a global counter (units then start in list order across the whole grid;
// the first unit costs no atomic round trip).
__device__ __forceinline__ int first_unit(const SweepArgs &) { return static_cast<int>(blockIdx.x); }

__device__ __forceinline__ int next_unit(const SweepArgs &a, int prev)
{
    return a.dyn ? static_cast<int>(gridDim.x + atomicAdd(a.dyn, 1u)) : prev + static_cast<int>(gridDim.x);
}

// A CTA's producer draws no more units: the last CTA of the launch (or of the
// step, in a persistent launch) to get here zeroes the counters for the next
// one (every other CTA has drawn its last index by then; kernel completion or
// the grid barrier publishes the reset).
__device__ __forceinline__ void units_done(const SweepArgs &a)
{
    if (!a.dyn)
        return;
    __threadfence();
    if (atomicAdd(a.dyn + 1, 1u) == gridDim.x - 1) {
        atomicExch(a.dyn, 0u);
        atomicExch(a.dyn + 1, 0u);
    }
}

// Bounded wait that also gives up as soon as another warp of the CTA has.
__device__ __forceinline__ bool wait_or_abort(uint64_t *bar, uint32_t parity, volatile int *abort_flag)
{
    if (mbar_try_wait(bar, parity))
        return true;
    const unsigned long long t0 = global_ns();
    while (!mbar_try_wait(bar, parity)) {
        if (*abort_flag)
            return false;
        if (global_ns() - t0 > kWaitLimitNs) {
            *abort_flag = 1;
            return false;
        }
    }
    return true;
}

// Grid-wide barrier of a persistent launch (all CTAs co-resident).  Thread 0
// publishes the CTA's stores (fence, and a proxy fence because the next step
// reads them through TMA), arrives on the counter and spins, bounded by
// kWaitLimitNs; on expiry the CTA's abort flag and the error word are set.  A
// CTA that has already aborted does not arrive, so the others time out too.
__device__ __forceinline__ bool grid_barrier(unsigned int *counter, unsigned int target, volatile int *abort_flag,
                                             int *err)
{
    __syncthreads();
    if (threadIdx.x == 0 && !*abort_flag) {
        __threadfence();
        asm volatile("fence.proxy.async.global;" ::: "memory");
        atomicAdd(counter, 1u);
        const unsigned long long t0 = global_ns();
        while (true) {
            unsigned int v;
            asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(counter) : "memory");
            if (v >= target)
                break;
            if (global_ns() - t0 > kWaitLimitNs) {
                *abort_flag = 1;
                atomicExch(err, static_cast<int>(kDevTimeoutBarrier));
                break;
            }
            __nanosleep(256);
        }
        asm volatile("fence.proxy.async.global;" ::: "memory");
    }
    __syncthreads();
    return *abort_flag == 0;
}

// Warp-specialised streaming sweep.  Warp NC is the TMA producer (one lane
// issues a plane load per iteration into ring slot it % S, completing on
// full[it % NB]); warps 0..NC-1 consume.  A consumer warp arrives on
// empty[j % NB] when it has finished iteration j (its newest plane and its
// centre plane, slot (j - rz) % S); the producer waits for empty of iteration
// it - NB before reusing that iteration's slot for iteration it.
//
// Work units come in list order, either statically (unit ui to CTA ui mod
// gridDim) or, with a.dyn, from a global counter that the producer draws from
// when it has issued the loads of its current unit (the first unit of CTA b is
// unit b), so that the units in flight stay a contiguous window
// of the list (neighbouring tiles at nearly the same planes: their shared halo
// rows are read from L2).  The producer records each unit's index for the
// consumers in uidx[] of its first iteration's barrier pair and ends a step
// with a sentinel iteration (index -1, a plain arrive, no load).
//
// YS = true (2D grids): the streaming axis is y.  A plane slot is one row of
// TX points (plus the x halo), the register queue holds the 2r+1 rows around
// the output row, and there is no middle axis; the update is the 2D one,
// ((x- + x+) + (y- + y+)) per offset, bit-identical to the 2D tile mode.
//
// OPT & kOptScalarOddX: the x-neighbour sums of odd offsets, whose operands
// straddle the thread's packed point pairs, as two scalar additions instead of
// one packed addition of re-paired registers (the same results bit for bit).
// OPT & kOptMixedY (BF16 storage): y-neighbour sums of two halo rows from the
// packed words by bf16_pair_sum (the same results bit for bit).
// OPT & kOptMixedU (BF16 wave): u^{n-1} - 2u by bf16_pair_sub, negated into the
// last fused multiply-add (the same results bit for bit).
template <int R, int EQ, int ST, bool HAS_Z, int NC, int PY, int D, int MINB, int TXT, bool YS = false, int OPT = 0>
__global__ void __launch_bounds__((NC + 1) * 32, MINB) k_stream(const SweepArgs a, const int slot_bytes)
{
    using St = Storage<ST>;
    constexpr bool SX = (OPT & kOptScalarOddX) != 0;
    constexpr bool MY = ST == GBST_BF16 && (OPT & kOptMixedY) != 0;
    constexpr bool MU = ST == GBST_BF16 && EQ == GBST_WAVE && (OPT & kOptMixedU) != 0;
    constexpr int NT = NC * 32;         // consumer threads
    constexpr int PX = St::PX;
    constexpr int ES = St::ES;
    constexpr int G = PX;               // x halo in elements (16 bytes)
    constexpr bool ZQ = HAS_Z || YS;    // a register queue along the streaming axis
    constexpr bool MID = !YS;           // y neighbours from the plane slot (3D, 2D tiles)
    constexpr int RZ = ZQ ? R : 0;      // radius along the streaming axis
    constexpr int QN = 2 * RZ + 1;      // register queue length
    constexpr int S = RZ + 1 + D;       // plane slots
    constexpr int NB = D + 1;           // barrier pairs (= loads in flight)
    constexpr int TX = TXT * PX;                 // tile width (points)
    constexpr int TY = (NT / TXT) * PY;          // tile height (rows; 1 when YS)
    static_assert(!YS || (TY == 1 && !HAS_Z), "y streaming: one-row tiles of a 2D grid");
    constexpr int ROW_BYTES = (TX + 2 * G) * ES; // one row of a plane slot
    // wave: kappa (FP32) and u^{n-1} of the centre plane, TX x TY each, per barrier pair
    constexpr int CK = TX * TY * 4;
    constexpr int CBYTES = CK + TX * TY * ES;
    constexpr int CSLOT = EQ == GBST_WAVE ? (CBYTES + 127) / 128 * 128 : 0;
    static_assert(R <= G, "x halo must cover the radius");
    static_assert(2 * NB * 8 + 16 + 4 * NB <= 256, "barrier header");
    static_assert(NT % TXT == 0, "tile shape");

    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *full = reinterpret_cast<uint64_t *>(smem);
    uint64_t *empty = full + NB;
    volatile int *abort_flag = reinterpret_cast<volatile int *>(empty + NB);
    volatile int *uidx = reinterpret_cast<volatile int *>(smem + 2 * NB * 8 + 16);  // unit of a unit's first iteration
    unsigned char *slots = smem + 256;
    unsigned char *cslots = slots + S * slot_bytes;  // wave centre-plane slots (NB of CSLOT bytes)

    // (a CTA without units still joins the grid barriers of a persistent launch)
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            mbar_init(&full[b], 1);
            mbar_init(&empty[b], NC);
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    // ------------------------------------------------------------ producer
    // One step's plane loads for this CTA's units; `it` counts iterations over
    // the whole launch (all steps), like the consumers' ring position.
    int it = 0;
    auto produce = [&](int parity) -> bool {
        // order the previous step's generic-proxy stores (made visible by the
        // grid barrier) before this thread's async-proxy (TMA) reads
        asm volatile("fence.proxy.async.global;" ::: "memory");
        for (int ui = first_unit(a); ui < a.nunits; ui = next_unit(a, ui)) {
            const Unit u = a.units[ui];
            const GridDev &g = a.grids[u.grid];
            const int bx = (u.tile % g.tiles_x) * TX, by = YS ? 0 : (u.tile / g.tiles_x) * TY;
            const CUtensorMap *map = &g.tmap[parity];
            const CUtensorMap *umap = &g.tmap_c[1 - parity];  // u^{n-1}, interior boxes
            const CUtensorMap *kmap = &g.tmap_k;              // kappa, interior boxes
            const uint32_t bytes = static_cast<uint32_t>(g.box_bytes);
            const int L = (u.z1 - u.z0) + 2 * RZ;
            for (int l = 0; l < L; ++l, ++it) {
                if (it >= NB && !wait_or_abort(&empty[it % NB], ((it / NB) - 1) & 1, abort_flag))
                    return false;
                if (l == 0)
                    uidx[it % NB] = ui;  // published by the arrive below (release)
                const bool centre = EQ == GBST_WAVE && l >= 2 * RZ;
                uint64_t *bar = &full[it % NB];
                mbar_arrive_expect_tx(bar, bytes + (centre ? CBYTES : 0));
                if (YS)  // row u.z0 - r + l (padded index u.z0 + l)
                    tma_load_plane(slots + (it % S) * slot_bytes, map, bar, bx, u.z0 + l, 0);
                else
                    tma_load_plane(slots + (it % S) * slot_bytes, map, bar, bx, by, u.z0 + l);
                if (centre) {
                    // centre plane of this iteration: interior z = z0 + l - 2rz, padded + rz
                    unsigned char *cs = cslots + (it % NB) * CSLOT;
                    const int zp = u.z0 + l - RZ;
                    if (YS) {
                        tma_load_plane(cs, kmap, bar, bx + G, zp, 0);
                        tma_load_plane(cs + CK, umap, bar, bx + G, zp, 0);
                    } else {
                        tma_load_plane(cs, kmap, bar, bx + G, by + R, zp);
                        tma_load_plane(cs + CK, umap, bar, bx + G, by + R, zp);
                    }
                }
            }
        }
        // sentinel iteration: no more units in this step
        if (it >= NB && !wait_or_abort(&empty[it % NB], ((it / NB) - 1) & 1, abort_flag))
            return false;
        uidx[it % NB] = -1;
        mbar_arrive(&full[it % NB]);
        ++it;
        units_done(a);
        return true;
    };

    // ----------------------------------------------------------- consumers
    const int tid = threadIdx.x;
    constexpr int PP = PX / 2;  // point pairs per row (packed FP32x2 arithmetic)
    float2 q[QN][PY][PP];       // z-queue of the thread's own points, by local plane index mod QN
    // iteration (plane) counter, kept as ring position, barrier index and phase parity
    int slot_n = 0;             // ring slot of the newest plane   (j mod S)
    int bar_i = 0;              // barrier pair of this iteration   (j mod NB)
    uint32_t par = 0;           // phase parity                     ((j / NB) & 1)
    auto advance = [&]() {
        slot_n = slot_n + 1 == S ? 0 : slot_n + 1;
        if (++bar_i == NB) {
            bar_i = 0;
            par ^= 1u;
        }
    };
    const float2 wc2 = make_float2(a.wc, a.wc);
    float2 w2[R + 1];
#pragma unroll
    for (int m = 0; m <= R; ++m)
        w2[m] = make_float2(a.w[m], a.w[m]);
    const float2 ls2 = make_float2(a.lscale, a.lscale);

    auto consume = [&](int parity, const float *srcval) -> bool {
        for (;;) {
            // the first iteration of the next unit, or the step's sentinel
            if (!wait_or_abort(&full[bar_i], par, abort_flag))
                return false;
            const int ui = uidx[bar_i];
            if (ui < 0) {
                __syncwarp();
                if (lane == 0)
                    mbar_arrive(&empty[bar_i]);
                advance();
                return true;
            }
            const Unit u = a.units[ui];
            // Copy the grid's descriptor into registers: the output stores below could
            // alias it, which would otherwise force a reload after every store.
            const GridDev *gp = a.grids + u.grid;
            const int tiles_x = gp->tiles_x;
            const int64_t nx = gp->nx, ny = gp->ny;
            const int64_t pitch = gp->pitch, rows = gp->rows, origin = gp->origin;
            unsigned char *__restrict__ outbase = static_cast<unsigned char *>(gp->buf[1 - parity]);
            const bool src_unit = (EQ == GBST_WAVE) && gp->has_src;
            const int src_x = gp->src_x, src_y = gp->src_y, src_z = gp->src_z;
            const float srcv = (EQ == GBST_WAVE && srcval) ? srcval[u.grid] : 0.0f;
            const float2 a2 = make_float2(gp->heat_a, gp->heat_a);
            const int tx = tid % TXT, ty = tid / TXT;
            const int x0 = (u.tile % tiles_x) * TX + tx * PX;
            const int y0 = YS ? 0 : (u.tile / tiles_x) * TY + ty * PY;
            constexpr int row_bytes = ROW_BYTES;
            const int own_off = ((MID ? R : 0) + ty * PY) * row_bytes + (G + tx * PX) * ES;
            const bool xfull = x0 + PX <= nx;
            bool row_ok[PY];
    #pragma unroll
            for (int r_ = 0; r_ < PY; ++r_)
                row_ok[r_] = (YS || y0 + r_ < ny) && x0 < nx;
            // running pointers to the thread's first row of the current output plane
            // output "planes" follow the streaming axis: planes (3D, 2D tiles) or rows (YS)
            const int64_t plane_elems = YS ? pitch : rows * pitch;
            unsigned char *optr = outbase + (origin + (static_cast<int64_t>(u.z0) * (YS ? 1 : rows) + y0) * pitch + x0) * ES;
            const int64_t row_stride = pitch * ES;

            // prologue: the 2*rz planes below the first output plane fill the queue
    #pragma unroll
            for (int k = 0; k < 2 * RZ; ++k) {
                if (!wait_or_abort(&full[bar_i], par, abort_flag))
                    return false;
                const unsigned char *nb = slots + slot_n * slot_bytes + own_off;
    #pragma unroll
                for (int r_ = 0; r_ < PY; ++r_) {
                    const uint4 v = lds128(nb + r_ * row_bytes);
    #pragma unroll
                    for (int pp = 0; pp < PP; ++pp)
                        q[k][r_][pp] = St::pair(v, pp);
                }
                __syncwarp();
                if (lane == 0)
                    mbar_arrive(&empty[bar_i]);
                advance();
            }

            const int nout = u.z1 - u.z0;
            for (int c0 = 0; c0 < nout; c0 += QN) {
    #pragma unroll
                for (int k = 0; k < QN; ++k) {
                    const int c = c0 + k;
                    if (c < nout) {
                        const int qn = (k + 2 * RZ) % QN;  // slot of the newest plane (constant after unrolling)
                        const int qc = (k + RZ) % QN;      // slot of the centre plane
                        const int zc = u.z0 + c;

                        float kap[PY][PX], um[PY][PX];
                        uint32_t umw[PY][PX / 2];  // MU: u^{n-1} as BF16 pairs
                        if (!wait_or_abort(&full[bar_i], par, abort_flag))
                            return false;
                        if (EQ == GBST_WAVE) {
                            // kappa and u^{n-1} of the centre plane, landed with this iteration's TMA
                            const unsigned char *cs = cslots + bar_i * CSLOT;
    #pragma unroll
                            for (int r_ = 0; r_ < PY; ++r_) {
                                const int e = (ty * PY + r_) * TX + tx * PX;
    #pragma unroll
                                for (int v = 0; v < PX / 4; ++v) {
                                    const uint4 kv = lds128(cs + (e + 4 * v) * 4);
                                    kap[r_][4 * v + 0] = __uint_as_float(kv.x);
                                    kap[r_][4 * v + 1] = __uint_as_float(kv.y);
                                    kap[r_][4 * v + 2] = __uint_as_float(kv.z);
                                    kap[r_][4 * v + 3] = __uint_as_float(kv.w);
                                }
                                const uint4 uv = lds128(cs + CK + e * ES);
                                if constexpr (MU) {
    #pragma unroll
                                    for (int pp = 0; pp < PX / 2; ++pp)
                                        umw[r_][pp] = word_of(uv, pp);
                                } else {
    #pragma unroll
                                    for (int i = 0; i < PX; ++i)
                                        um[r_][i] = St::get(uv, i);
                                }
                            }
                        }
                        {
                            const unsigned char *nb = slots + slot_n * slot_bytes + own_off;
    #pragma unroll
                            for (int r_ = 0; r_ < PY; ++r_) {
                                const uint4 v = lds128(nb + r_ * row_bytes);
    #pragma unroll
                                for (int pp = 0; pp < PP; ++pp)
                                    q[qn][r_][pp] = St::pair(v, pp);
                            }
                        }

                        const int slot_c = slot_n >= RZ ? slot_n - RZ : slot_n - RZ + S;
                        const unsigned char *cb = slots + slot_c * slot_bytes + own_off;
                        uint4 ylo[R], yhi[R], xl[PY], xr[PY];
                        if (MID) {
    #pragma unroll
                            for (int m = 1; m <= R; ++m) {
                                ylo[m - 1] = lds128(cb - m * row_bytes);
                                yhi[m - 1] = lds128(cb + (PY - 1 + m) * row_bytes);
                            }
                        }
    #pragma unroll
                        for (int r_ = 0; r_ < PY; ++r_) {
                            xl[r_] = load_left<ST, R>(cb + r_ * row_bytes - 16);
                            xr[r_] = load_right<ST, R>(cb + r_ * row_bytes + 16);
                        }

                        // element e in [-G, PX+G) of centre row r_: own points or the x-halo chunks
                        auto xel = [&](int r_, int e) -> float {
                            if (e < 0)
                                return St::get(xl[r_], PX + e);
                            if (e >= PX)
                                return St::get(xr[r_], e - PX);
                            return (e & 1) ? q[qc][r_][e >> 1].y : q[qc][r_][e >> 1].x;
                        };
                        // pair pp of centre-plane row `row` (relative to the thread's first row)
                        auto yrow = [&](int row, int pp) -> float2 {
                            if (row < 0)
                                return St::pair(ylo[-row - 1], pp);
                            if (row >= PY)
                                return St::pair(yhi[row - PY], pp);
                            return q[qc][row][pp];
                        };
                        // Per point: t_m = ((x-m + x+m) + (y-m + y+m)) + (z-m + z+m) for every m
                        // (independent of each other), then s = w0*ndim*c, s = fma(w_m, t_m, s)
                        // for m = 1..r.  The dependent chain is r + 3 deep instead of 3r + 1.
                        float2 sv[PY][PP];
    #pragma unroll
                        for (int r_ = 0; r_ < PY; ++r_)
    #pragma unroll
                            for (int pp = 0; pp < PP; ++pp)
                                sv[r_][pp] = __fmul2_rn(wc2, q[qc][r_][pp]);
    #pragma unroll
                        for (int m = 1; m <= R; ++m) {
    #pragma unroll
                            for (int r_ = 0; r_ < PY; ++r_) {
    #pragma unroll
                                for (int pp = 0; pp < PP; ++pp) {
                                    const int e = 2 * pp;
                                    const float2 xm = make_float2(xel(r_, e - m), xel(r_, e + 1 - m));
                                    const float2 xp = make_float2(xel(r_, e + m), xel(r_, e + 1 + m));
                                    float2 t;
                                    if (SX && (m & 1)) {
                                        t.x = __fadd_rn(xm.x, xp.x);
                                        t.y = __fadd_rn(xm.y, xp.y);
                                    } else {
                                        t = __fadd2_rn(xm, xp);
                                    }
                                    if (MID) {
                                        float2 ys;
                                        if (MY && r_ - m < 0 && r_ + m >= PY)
                                            ys = bf16_pair_sum(word_of(ylo[m - r_ - 1], pp), word_of(yhi[r_ + m - PY], pp));
                                        else
                                            ys = __fadd2_rn(yrow(r_ - m, pp), yrow(r_ + m, pp));
                                        t = __fadd2_rn(t, ys);
                                    }
                                    if (ZQ)
                                        t = __fadd2_rn(t, __fadd2_rn(q[(qc - m + 2 * QN) % QN][r_][pp], q[(qc + m) % QN][r_][pp]));
                                    sv[r_][pp] = __ffma2_rn(w2[m], t, sv[r_][pp]);
                                }
                            }
                        }
                        float o[PY][PX];
    #pragma unroll
                        for (int r_ = 0; r_ < PY; ++r_) {
    #pragma unroll
                            for (int pp = 0; pp < PP; ++pp) {
                                const float2 cv = q[qc][r_][pp];
                                float2 ov;
                                if (EQ == GBST_HEAT) {
                                    ov = __ffma2_rn(a2, sv[r_][pp], cv);
                                } else if constexpr (MU) {
                                    const float2 k2 = make_float2(kap[r_][2 * pp], kap[r_][2 * pp + 1]);
                                    const float2 n2 = bf16_pair_sub(umw[r_][pp], __fadd2_rn(cv, cv));
                                    ov = __ffma2_rn(k2, __fmul2_rn(ls2, sv[r_][pp]), make_float2(-n2.x, -n2.y));
                                } else {
                                    const float2 k2 = make_float2(kap[r_][2 * pp], kap[r_][2 * pp + 1]);
                                    const float2 t2 = __fadd2_rn(__fadd2_rn(cv, cv),
                                                                 make_float2(-um[r_][2 * pp], -um[r_][2 * pp + 1]));
                                    ov = __ffma2_rn(k2, __fmul2_rn(ls2, sv[r_][pp]), t2);
                                }
                                o[r_][2 * pp] = ov.x;
                                o[r_][2 * pp + 1] = ov.y;
                            }
                        }
                        // all shared-memory reads of this iteration are done: release the planes
                        __syncwarp();
                        if (lane == 0)
                            mbar_arrive(&empty[bar_i]);
                        advance();

                        if (src_unit && zc == (YS ? src_y : src_z)) {
                            const int sr = YS ? 0 : src_y - y0, si = src_x - x0;
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
                            if (row_ok[r_]) {
                                unsigned char *op = optr + r_ * row_stride;
                                if (xfull) {
                                    *reinterpret_cast<uint4 *>(op) = St::pack(o[r_]);
                                } else {
    #pragma unroll
                                    for (int i = 0; i < PX; ++i)
                                        if (x0 + i < nx)
                                            St::store1(op + i * ES, o[r_][i]);
                                }
                            }
                        }
                        optr += plane_elems * ES;
                    }
                }
            }
        }
        return true;
    };

    // --------------------------------------------------------------- steps
    // nsteps == 1: one sweep.  nsteps > 1 (persistent launch, all CTAs
    // co-resident): a grid-wide barrier separates the steps, the parity flips.
    bool ok = true;
    for (int step = 0; step < a.nsteps; ++step) {
        const int parity = a.parity ^ (step & 1);
        const float *srcval = a.srcval ? a.srcval + static_cast<int64_t>(step) * a.ngrids : nullptr;
        if (warp == NC) {
            if (lane == 0 && ok)
                ok = produce(parity);
        } else if (ok) {
            ok = consume(parity, srcval);
            if (!ok)  // a wait gave up (the producer may have left already): report it here
                atomicCAS(a.err, 0, static_cast<int>(kDevTimeoutTma));
        }
        if (step + 1 < a.nsteps &&
            !grid_barrier(a.barrier, static_cast<unsigned int>(step + 1) * gridDim.x + a.barrier_extra, abort_flag,
                          a.err))
            break;
    }
    if (warp == NC && lane == 0 && *abort_flag) {
        atomicCAS(a.err, 0, static_cast<int>(kDevTimeoutTma));
        // let the loads already issued land before the CTA can exit (short bound)
        for (int k = it - NB < 0 ? 0 : it - NB; k < it; ++k) {
            const unsigned long long t0 = global_ns();
            while (!mbar_try_wait(&full[k % NB], (k / NB) & 1) && global_ns() - t0 < 50000000ull) {
            }
        }
    }
}

}  // namespace

// ---- variant tables ----------------------------------------------------------
using KernelFn = void (*)(const SweepArgs, const int);

struct Entry {
    StreamVariant v;
    KernelFn fn;
};

template <int R, int EQ, int ST, bool HZ, int NC, int PY, int D, int MINB, int TXT, bool YS = false, int OPT = 0>
constexpr Entry entry()
{
    return Entry{StreamVariant{R, EQ, ST, HZ, NC * 32, PY, D, MINB, TXT, 1, YS, 1, OPT},
                 &k_stream<R, EQ, ST, HZ, NC, PY, D, MINB, TXT, YS, OPT>};
}

// both equations for one radius, storage, dimensionality and shape
#define GBST_EQS(R, ST, HZ, NC, PY, D, MINB, TXT) \
    entry<R, GBST_HEAT, ST, HZ, NC, PY, D, MINB, TXT>(), entry<R, GBST_WAVE, ST, HZ, NC, PY, D, MINB, TXT>()
// 2D, streaming along y: one consumer warp, one-row tiles of 32 x 16 bytes
#define GBST_EQS_YS(R, ST, D, MINB)                                    \
    entry<R, GBST_HEAT, ST, false, 1, 1, D, MINB, 32, true>(),        \
        entry<R, GBST_WAVE, ST, false, 1, 1, D, MINB, 32, true>()

}  // namespace sweep
}  // namespace gbst
