// 3x3x3 convolution of a channels-last 16-channel BF16 tensor on the 5th-
// generation tensor cores (tcgen05.mma, accumulators in tensor memory),
// zero padding, 16 output channels (fewer are zero-padded weights).
//
// Implicit GEMM per output row segment: D[128 points x 16 co] = sum over the 27
// taps of A_tap[128 points x 16 ci] B_tap[16 ci x 16 co].  A CTA owns 128
// consecutive x points of RY = 4 rows and marches along z.  For every input
// plane a TMA load brings rows y0-1..y0+RY, x0-1..x0+128 (out of range ->
// zeros, which is the zero padding) as one box of 16 channels in the 32-byte
// swizzled layout, a K-major tcgen05 operand whose rows are the points' 32
// bytes (see Geo).  A_tap of row r is then just a shifted view of the plane
// slot (start address + (r + dy) * row + dx * 32 bytes), no data movement per
// tap.  The weights of all taps sit in shared memory, K-major and unswizzled.
//
// Input-stationary order: when input plane p has landed, its taps are issued
// at once into the three outputs that read it (p + 1 through dz = 0, p through
// dz = 1, p - 1 through dz = 2), which completes output p - 1, and the plane
// is released right after; the ring of NS slots keeps NS - 1 planes of
// prefetch in flight.  The three outputs share the A operand of a tap
// (dy, dx), so one MMA with N = 48 computes all three: output o accumulates in
// tensor-memory slot o mod 3 (16 columns per row), and the weights of a tap are
// stored as five 16-row blocks in dz order 2, 1, 0, 2, 1, so that the three
// consecutive blocks starting at block 2 - ((p + 1) mod 3) line up with slots
// 0, 1, 2.  An M = 128 MMA reads its 4 KB A tile from shared memory whatever
// its N (about 32 cycles at 128 bytes per cycle, plus N / 4 for B), so the
// N = 48 form does the work of three N = 16 MMAs in 44 instead of 117 cycles.
// All MMAs accumulate; the epilogue zeroes a slot right after reading it.
// At a unit's first two and last two planes some of the three outputs lie
// outside the unit; those planes issue one N = 16 MMA per valid output.
//
// Warp roles: warps 0-7 epilogue (warp w reads tensor-memory lanes
// 32 (w & 3) .. +31 = points, channels 8 (w >> 2) .. +7 of each row), warp 8
// TMA producer (one lane), warp 9 allocates the tensor memory and issues the
// MMAs (the whole warp runs the loop, elect.sync picks the issuing lane: a
// loop run by one lane alone issued an MMA only every 144 cycles).
// Pipelines: input plane ring (full / empty mbarriers; a tcgen05.commit frees
// a plane once the MMAs reading it are done) and the three accumulator slots
// (tfull: commit after an output's last taps; tempty: the epilogue warps,
// after reading and zeroing the slot).
// Every wait is bounded; on expiry the CTA sets the error word, lets issued
// work finish (bounded) and releases its tensor memory.
#pragma once

#include <type_traits>

#include "gbst_internal.h"

namespace gbst {
namespace convtc {

constexpr int TXP = 128;                 // output points per CTA row segment (MMA M)
constexpr int RY = 4;                    // output rows per CTA (independent accumulation chains)
constexpr int BOXY = RY + 2;             // input rows per plane (y halo 1 each side)
constexpr int NS = 3;                    // plane slots: two planes of prefetch
constexpr int NACC = 3;                  // accumulator slots: output o in slot o mod 3
constexpr int ROWCOLS = NACC * 16;       // tensor-memory columns of one output row (the N = 48 MMA)
constexpr int TCOLS = 256;               // allocated columns (RY x 48 = 192 used; two CTAs per SM fill the 512)
constexpr int WBLK = 5;                  // weight blocks per tap: dz = 2, 1, 0, 2, 1
constexpr int WHALF = WBLK * 16 * 16;    // bytes of one 8-channel K half of a tap: [80 rows][8 ci] BF16
constexpr int WTAP = 2 * WHALF;          // bytes of one tap
constexpr int HDR = 256;                 // barriers and flags
constexpr int NEPI = 8;                  // epilogue warps: lane quadrant w & 3, channels 8 (w >> 2) ..
constexpr int NTHREADS = (NEPI + 2) * 32;
constexpr int ZCH = 32;                  // output planes per work unit

// Plane geometry by input width.  CIN = 16: one box of all 16 channels per plane
// (32-byte rows) in the 32-byte swizzled K-major layout, so the K = 16 operand of
// a tap is one 32-byte row per point; rows of 136 points start on 256-byte pattern
// boundaries (two boxes of 8 channels, 16-byte rows each half an L2 sector, made
// twice the L2 requests and bounded the layer).  Nine (dy, dx) taps.  CIN = 8 (16
// bytes per point, unswizzled): one box, and the K = 16 operand pairs a point with
// its x neighbour (the second core matrix along K starts 16 bytes later), so taps
// dx = -1 and 0 form one MMA and dx = +1 another (its second K half has zero
// weights): six taps (dy, pair | single).  Its rows carry two extra points so that
// the single tap's second half stays inside the row.
template <int CIN>
struct Geo;
template <>
struct Geo<16> {
    static constexpr int BOXX = 136;                               // input points per row (x halo 1 | 7)
    static constexpr int ROWB = BOXX * 32;                         // bytes of one row, 16 channels
    static constexpr int SLOT = (BOXY * ROWB + 1023) / 1024 * 1024;
    static constexpr bool SW32 = true;                             // 32-byte swizzle
    static constexpr int LBO_A = 16;                               // (unused by a swizzled K-major operand)
    static constexpr int NTAP = 9;
    __host__ __device__ static constexpr int a_off(int t, int r) { return (r + t / 3) * ROWB + (t % 3) * 32; }
};
template <>
struct Geo<8> {
    static constexpr int BOXX = TXP + 4;
    static constexpr int ROWB = BOXX * 16;
    static constexpr int SLOT = (BOXY * ROWB + 127) / 128 * 128;
    static constexpr bool SW32 = false;
    static constexpr int LBO_A = 16;                               // K half 2: the next point
    static constexpr int NTAP = 6;
    __host__ __device__ static constexpr int a_off(int t, int r) { return (r + t / 2) * ROWB + (t % 2) * 32; }
};
// CIN = 8 through a blocked view of the input, for rows of a multiple of 32 points:
// the tensor map sees each row as blocks of 32 points x 8 channels (512 contiguous
// bytes), and a box of 6 blocks from the block before x0 lands as rows of 192
// points, the same unswizzled layout as Geo<8> (x0 - 1 at point 31 of a row).  Each
// TMA box row is then 512 bytes instead of one point's 16, a fraction of the L2
// requests (one per point row had bounded the layer).
struct GeoB8 {
    static constexpr int BOXX = 192;
    static constexpr int ROWB = BOXX * 16;
    static constexpr int SLOT = BOXY * ROWB;
    static constexpr int BLOCKS = BOXX / 32;                       // blocks of 32 points per box row
    static constexpr bool SW32 = false;
    static constexpr int LBO_A = 16;
    static constexpr int NTAP = 6;
    __host__ __device__ static constexpr int a_off(int t, int r)
    {
        return (r + t / 2) * ROWB + 31 * 16 + (t % 2) * 32;
    }
};
template <int CIN, bool BLK>
using GeoOf = typename std::conditional<BLK, GeoB8, Geo<CIN>>::type;

template <int CIN, bool BLK = false>
constexpr int tc_smem()
{
    using G = GeoOf<CIN, BLK>;
    return HDR + G::NTAP * WTAP + (G::SW32 ? 1024 : 0) + NS * G::SLOT;
}

__device__ __forceinline__ uint32_t sa(const void *p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }

__device__ __forceinline__ unsigned long long now_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void bar_init(uint64_t *b, uint32_t n)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(sa(b)), "r"(n) : "memory");
}

__device__ __forceinline__ void bar_arrive(uint64_t *b)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(sa(b)) : "memory");
}

__device__ __forceinline__ void bar_expect(uint64_t *b, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(sa(b)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool bar_try(uint64_t *b, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(sa(b)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait; gives up when another thread of the CTA has given up.
__device__ __forceinline__ bool bar_wait(uint64_t *b, uint32_t parity, volatile int *abort_flag)
{
    if (bar_try(b, parity))
        return true;
    const unsigned long long t0 = now_ns();
    while (!bar_try(b, parity)) {
        if (*abort_flag)
            return false;
        if (now_ns() - t0 > kWaitLimitNs) {
            *abort_flag = 1;
            return false;
        }
    }
    return true;
}

__device__ __forceinline__ void tma_load_4d(void *dst, const CUtensorMap *map, uint64_t *bar, int c, int x, int y,
                                            int z)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(sa(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c), "r"(x), "r"(y), "r"(z), "r"(sa(bar))
        : "memory");
}

// Shared-memory matrix descriptor (K-major, no swizzle) as two 32-bit halves,
// so that a per-tap offset is one 32-bit add on the low half (start address
// field; offsets stay inside the operand).  lbo: bytes between core matrices
// along K, sbo: bytes between 8-row groups along M / N.
__device__ __forceinline__ uint32_t sdesc_lo(uint32_t addr, uint32_t lbo)
{
    return ((addr >> 4) & 0x3FFFu) | (((lbo >> 4) & 0x3FFFu) << 16);
}
constexpr uint32_t sdesc_hi(uint32_t sbo) { return ((sbo >> 4) & 0x3FFFu) | (1u << 14); }
// The same for a K-major operand in the 32-byte swizzled layout (rows of 32 bytes, the
// two 16-byte halves of a row exchanged in rows 4-7 of every 256 bytes, as a TMA load
// with 32-byte swizzle writes it); the start address may sit anywhere in the pattern.
constexpr uint32_t sdesc_hi_sw32(uint32_t sbo) { return sdesc_hi(sbo) | (6u << 29); }

// Instruction descriptor of kind::f16: BF16 A and B (K-major), FP32 D, M = 128, N = n.
constexpr uint32_t idesc_bf16(uint32_t n)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((n >> 3) << 17) | ((128u >> 4) << 24);
}

// D[tmem] += A B, issued by one lane that elect.sync picks: the whole (converged)
// warp executes the statement.  Descriptors as 32-bit halves.
__device__ __forceinline__ void mma_bf16_warp(uint32_t d_tmem, uint32_t alo, uint32_t ahi, uint32_t blo,
                                              uint32_t bhi, uint32_t idesc)
{
    asm volatile(
        "{\n\t.reg .pred e;\n\t.reg .b32 l;\n\t.reg .b64 da, db;\n\t"
        "elect.sync l|e, 0xffffffff;\n\t"
        "mov.b64 da, {%1, %2};\n\t"
        "mov.b64 db, {%3, %4};\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], da, db, %5, 1;\n\t}" ::"r"(d_tmem),
        "r"(alo), "r"(ahi), "r"(blo), "r"(bhi), "r"(idesc));
}

// tcgen05.commit of the MMAs issued so far, from one elected lane of the converged warp.
__device__ __forceinline__ void mma_commit_warp(uint64_t *bar)
{
    asm volatile(
        "{\n\t.reg .pred e;\n\t.reg .b32 l;\n\t"
        "elect.sync l|e, 0xffffffff;\n\t"
        "@e tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n\t}" ::"r"(sa(bar))
        : "memory");
}

// Zero 8 consecutive FP32 columns of the warp's 32 lanes (no wait).
__device__ __forceinline__ void tmem_zero8(uint32_t taddr)
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %1, %1, %1, %1, %1, %1, %1};" ::"r"(taddr),
                 "r"(0u)
                 : "memory");
}

__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// Four loads of 8 columns (one per output row) and a single wait: the values
// pass through the wait (as read-write operands of an empty statement after
// it), so no use can be scheduled before the loads have completed.
__device__ __forceinline__ void tmem_ld8x4(uint32_t taddr, uint32_t stride, float (&v)[4][8])
{
    uint32_t r[4][8];
#pragma unroll
    for (int q = 0; q < 4; ++q)
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                     : "=r"(r[q][0]), "=r"(r[q][1]), "=r"(r[q][2]), "=r"(r[q][3]), "=r"(r[q][4]), "=r"(r[q][5]),
                       "=r"(r[q][6]), "=r"(r[q][7])
                     : "r"(taddr + q * stride));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        asm volatile(""
                     : "+r"(r[q][0]), "+r"(r[q][1]), "+r"(r[q][2]), "+r"(r[q][3]), "+r"(r[q][4]), "+r"(r[q][5]),
                       "+r"(r[q][6]), "+r"(r[q][7]));
#pragma unroll
        for (int i = 0; i < 8; ++i)
            v[q][i] = __uint_as_float(r[q][i]);
    }
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Work unit u -> (row group y0, x chunk, z chunk); z chunk outermost so that
// the CTAs of one wave hold neighbouring rows of the same planes (halo rows
// shared in L2).
struct UnitMap {
    int nxc, nzc, nyc, nz;
    __device__ void decode(int u, int &y0, int &x0, int &z0, int &z1) const
    {
        const int xc = u % nxc;
        const int rest = u / nxc;
        y0 = (rest % nyc) * RY;
        const int zc = rest / nyc;
        x0 = xc * TXP;
        z0 = zc * ZCH;
        z1 = min(nz, z0 + ZCH);
    }
};

}  // namespace convtc
}  // namespace gbst
