// Learned closure for a 2x-coarsened acoustic-wave solve: a 3-layer 3x3x3
// convolutional network (C_in = 4 -> 16 -> 16 -> 1, GELU), BF16 weights and
// activations, FP32 accumulation on the tensor cores (mma.sync m16n8k16), with
// its backward pass and an Adam optimiser.  The paper has no learned part.
//
// Network (per coarse step, inputs scaled by s, c_n = c / c_ref):
//   x  = s (u+, u^n, c_n^2 u+, c_n^2 u^n)    u+ = the plain coarse step
//   z1 = conv1(x) + b1,  y1 = GELU(z1)
//   z2 = conv2(y1) + b2, y2 = GELU(z2)
//   o  = conv3(y2) + b3                       u+ += o / t  (t: output scale)
// Training minimises mean((o - t (u_ref - u+))^2) over all points.
//
// Layouts: every activation is channels-last BF16 with 16 channels (inputs and
// the 1-channel gradient padded with zeros); weights are kept in FP32 (master,
// order [co][ci][dz][dy][dx] per layer, then the biases) and converted to BF16
// [tap][co][16] for the forward convolutions and to the flipped, transposed
// [tap][ci][16] for the data gradient.
#include <cmath>
#include <vector>

#include "conv_tc.cuh"
#include "gbst_internal.h"

namespace gbst {
namespace {

constexpr int CH = 16;               // channels of every stored activation
constexpr int TXC = 32, TYC = 4;     // output tile of a CTA (x, y)
constexpr int HX = TXC + 2, HY = TYC + 2;
constexpr int PLANE_PTS = HX * HY;   // halo tile points per plane
constexpr int PLANE_BYTES = PLANE_PTS * 32;
constexpr int NSLOT = 4;             // plane ring: z-1, z, z+1 and one prefetch
constexpr int NTHR = 256;            // 8 warps; warp w: row w/2, 16-point segment w%2
constexpr int ZCHUNK = 16;           // output planes per CTA

enum Epi { EPI_GELU = 0, EPI_LINEAR_F32 = 1, EPI_DGELU = 2, EPI_LINEAR_BF16 = 3 };

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Row-swizzled byte offset of half `half` (8 channels, 16 B) of row `row` in a
// 32-byte-row matrix: the halves of every other group of 4 rows are swapped so
// that the 8 rows an ldmatrix phase reads fall on distinct banks.
__device__ __forceinline__ int swz(int row, int half) { return row * 32 + ((half ^ ((row >> 2) & 1)) << 4); }

__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t &r0, uint32_t &r1, uint32_t &r2, uint32_t &r3)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(addr));
}

__device__ __forceinline__ void ldsm_x4_t(uint32_t addr, uint32_t &r0, uint32_t &r1, uint32_t &r2, uint32_t &r3)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(addr));
}

__device__ __forceinline__ void ldsm_x2(uint32_t addr, uint32_t &r0, uint32_t &r1)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0, %1}, [%2];" : "=r"(r0), "=r"(r1) : "r"(addr));
}

__device__ __forceinline__ void mma16816(float (&c)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3, uint32_t b0,
                                         uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, bool valid)
{
    const int n = valid ? 16 : 0;  // 0: zero-fill, nothing read
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// GELU(x) = x Phi(x) of the forward convolutions.  Phi from the complementary
// error function approximation of Abramowitz & Stegun, Handbook of
// Mathematical Functions, formula 7.1.26 (|error| <= 1.5e-7 in erf):
// erfc(z) ~ t (a1 + t (a2 + t (a3 + t (a4 + t a5)))) exp(-z^2), t = 1 / (1 + p z),
// with z = |x| / sqrt(2), so that 1 - Phi(|x|) = erfc(z) / 2.  Below, p is divided
// by sqrt(2) and the a_k by 2; the exponential is 2^(-x^2 log2(e) / 2).  In FP32
// the result is within 1.8e-7 max(1, |x|) of the exact GELU.  Two special-function
// instructions (reciprocal, exp2) and packed FP32x2 arithmetic for two values.
constexpr float kGp = 0.231641900f;                   // p / sqrt(2), p = 0.3275911
constexpr float kGa1 = 0.127414796f, kGa2 = -0.142248368f, kGa3 = 0.710706871f, kGa4 = -0.726576014f,
                kGa5 = 0.530702715f;                  // a_k / 2
constexpr float kGe = -0.721347520f;                  // -log2(e) / 2
__device__ __forceinline__ float rcp_approx(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float2 gelu2(float2 v)
{
    const float2 ax = make_float2(fabsf(v.x), fabsf(v.y));
    const float2 d = __ffma2_rn(make_float2(kGp, kGp), ax, make_float2(1.0f, 1.0f));
    const float2 t = make_float2(rcp_approx(d.x), rcp_approx(d.y));
    float2 q = __ffma2_rn(t, make_float2(kGa5, kGa5), make_float2(kGa4, kGa4));
    q = __ffma2_rn(t, q, make_float2(kGa3, kGa3));
    q = __ffma2_rn(t, q, make_float2(kGa2, kGa2));
    q = __ffma2_rn(t, q, make_float2(kGa1, kGa1));
    q = __fmul2_rn(q, t);
    const float2 sx = __fmul2_rn(__fmul2_rn(v, make_float2(kGe, kGe)), v);
    const float2 h = __fmul2_rn(q, make_float2(ex2_approx(sx.x), ex2_approx(sx.y)));  // 1 - Phi(|x|)
    const float2 phi = make_float2(v.x >= 0.0f ? 1.0f - h.x : h.x, v.y >= 0.0f ? 1.0f - h.y : h.y);
    return __fmul2_rn(v, phi);
}
__device__ __forceinline__ float gelu(float x) { return gelu2(make_float2(x, 0.0f)).x; }
// GELU'(x) of the backward pass (exact erf form).
__device__ __forceinline__ float gelu_grad(float x)
{
    return 0.5f * (1.0f + erff(x * 0.70710678118654752f)) + x * 0.39894228040143268f * expf(-0.5f * x * x);
}

struct Dims {
    int nx, ny, nz;
};

// Load plane z (interior index; outside [0, nz) -> zeros) of the halo tile at
// (x0-1 .. x0+TXC, y0-1 .. y0+TYC) of a channels-last 16-channel BF16 tensor.
__device__ __forceinline__ void load_plane(unsigned char *slot, const __nv_bfloat16 *in, Dims d, int x0, int y0, int z)
{
    const bool zin = z >= 0 && z < d.nz;
    for (int idx = threadIdx.x; idx < PLANE_PTS * 2; idx += NTHR) {
        const int pt = idx >> 1, half = idx & 1;
        const int gx = x0 - 1 + pt % HX, gy = y0 - 1 + pt / HX;
        const bool valid = zin && gx >= 0 && gx < d.nx && gy >= 0 && gy < d.ny;
        const __nv_bfloat16 *src =
            valid ? in + ((static_cast<int64_t>(z) * d.ny + gy) * d.nx + gx) * CH + half * 8 : in;
        cp_async16(smem_addr(slot + swz(pt, half)), src, valid);
    }
}

// Load plane z of the interior tile (no halo) of a 16-channel tensor.
__device__ __forceinline__ void load_tile(unsigned char *dst, const __nv_bfloat16 *in, Dims d, int x0, int y0, int z)
{
    for (int idx = threadIdx.x; idx < TXC * TYC * 2; idx += NTHR) {
        const int pt = idx >> 1, half = idx & 1;
        const int gx = x0 + pt % TXC, gy = y0 + pt / TXC;
        const bool valid = gx < d.nx && gy < d.ny;
        const __nv_bfloat16 *src =
            valid ? in + ((static_cast<int64_t>(z) * d.ny + gy) * d.nx + gx) * CH + half * 8 : in;
        cp_async16(smem_addr(dst + swz(pt, half)), src, valid);
    }
}

struct ConvArgs {
    const __nv_bfloat16 *in;   // [z][y][x][16]
    const __nv_bfloat16 *wt;   // [27][COUT][16] (tap = (dz*3 + dy)*3 + dx)
    const float *bias;         // [COUT] or null
    __nv_bfloat16 *out;        // EPI_GELU / EPI_DGELU: [z][y][x][16]
    __nv_bfloat16 *zout;       // EPI_GELU: pre-activations (optional)
    const __nv_bfloat16 *aux;  // EPI_DGELU: pre-activations of the layer below
    float *out_f32;            // EPI_LINEAR_F32: channel 0, dense [z][y][x]
    float oscale;              // EPI_LINEAR_F32: factor on the output (1 for the network units)
    Dims d;
    int cout_valid;            // output channels that are real (the rest are written as 0)
};

// 3x3x3 convolution, zero padding, one CTA per (32 x 4) column and ZCHUNK planes.
template <int COUT, int EPI>
__global__ void __launch_bounds__(NTHR) k_conv(const ConvArgs a)
{
    constexpr int NT = COUT / 8;  // n-tiles of 8 output channels
    extern __shared__ __align__(128) unsigned char sm[];
    unsigned char *wsm = sm;                               // 27 * COUT rows of 32 B
    unsigned char *ring = sm + 27 * COUT * 32;             // NSLOT plane slots
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int tiles_x = (a.d.nx + TXC - 1) / TXC;
    const int x0 = (blockIdx.x % tiles_x) * TXC, y0 = (blockIdx.x / tiles_x) * TYC;
    const int z0 = blockIdx.y * ZCHUNK;
    const int z1 = min(a.d.nz, z0 + ZCHUNK);

    for (int idx = tid; idx < 27 * COUT * 2; idx += NTHR) {
        const int row = idx >> 1, half = idx & 1;
        cp_async16(smem_addr(wsm + swz(row, half)), a.wt + row * 16 + half * 8, true);
    }
    load_plane(ring + 0 * PLANE_BYTES, a.in, a.d, x0, y0, z0 - 1);
    load_plane(ring + 1 * PLANE_BYTES, a.in, a.d, x0, y0, z0);
    cp_commit();
    load_plane(ring + 2 * PLANE_BYTES, a.in, a.d, x0, y0, z0 + 1);
    cp_commit();

    const int wy = warp >> 1, ws = warp & 1;
    const int m = lane >> 3, r = lane & 7;
    const int a_pt = r + 8 * (m & 1), a_half = m >> 1;  // A fragment rows (points) / channel half
    const int g = lane >> 2, q = lane & 3;
    const int y = y0 + wy;

    for (int z = z0; z < z1; ++z) {
        // planes z-1, z, z+1 must be resident; prefetch z+2 into the free slot
        load_plane(ring + ((z + 2 - z0 + 1) % NSLOT) * PLANE_BYTES, a.in, a.d, x0, y0, z + 2);
        cp_commit();
        cp_wait<1>();
        __syncthreads();

        float acc[NT][4];
#pragma unroll
        for (int t = 0; t < NT; ++t)
#pragma unroll
            for (int k = 0; k < 4; ++k)
                acc[t][k] = 0.f;
#pragma unroll
        for (int kz = 0; kz < 3; ++kz) {
            const unsigned char *slot = ring + ((z + kz - 1 - z0 + 1) % NSLOT) * PLANE_BYTES;
#pragma unroll
            for (int ky = 0; ky < 3; ++ky) {
#pragma unroll
                for (int kx = 0; kx < 3; ++kx) {
                    const int tap = (kz * 3 + ky) * 3 + kx;
                    const int pt = (wy + ky) * HX + ws * 16 + a_pt + kx;
                    uint32_t a0, a1, a2, a3;
                    ldsm_x4(smem_addr(slot + swz(pt, a_half)), a0, a1, a2, a3);
                    if (NT == 2) {
                        uint32_t b0, b1, b2, b3;
                        ldsm_x4(smem_addr(wsm + swz(tap * COUT + (m >> 1) * 8 + r, m & 1)), b0, b1, b2, b3);
                        mma16816(acc[0], a0, a1, a2, a3, b0, b1);
                        mma16816(acc[NT - 1], a0, a1, a2, a3, b2, b3);
                    } else {
                        uint32_t b0, b1;
                        ldsm_x2(smem_addr(wsm + swz(tap * COUT + r, m & 1)), b0, b1);
                        mma16816(acc[0], a0, a1, a2, a3, b0, b1);
                    }
                }
            }
        }

        // epilogue: C rows = points g, g+8 of the warp's segment; cols = channels 8t + 2q, +1
#pragma unroll
        for (int half8 = 0; half8 < 2; ++half8) {
            const int x = x0 + ws * 16 + g + 8 * half8;
            if (x >= a.d.nx || y >= a.d.ny)
                continue;
            const int64_t p = (static_cast<int64_t>(z) * a.d.ny + y) * a.d.nx + x;
#pragma unroll
            for (int t = 0; t < NT; ++t) {
                const int c = 8 * t + 2 * q;
                float v0 = acc[t][2 * half8], v1 = acc[t][2 * half8 + 1];
                if (EPI == EPI_LINEAR_F32) {
                    if (c == 0)
                        a.out_f32[p] = (v0 + a.bias[0]) * a.oscale;
                } else if (EPI == EPI_GELU) {
                    v0 += a.bias[c];
                    v1 += a.bias[c + 1];
                    if (c >= a.cout_valid)
                        v0 = 0.f;
                    if (c + 1 >= a.cout_valid)
                        v1 = 0.f;
                    if (a.zout)
                        *reinterpret_cast<__nv_bfloat162 *>(a.zout + p * CH + c) = __floats2bfloat162_rn(v0, v1);
                    const float2 g = gelu2(make_float2(v0, v1));
                    *reinterpret_cast<__nv_bfloat162 *>(a.out + p * CH + c) = __floats2bfloat162_rn(g.x, g.y);
                } else if (EPI == EPI_LINEAR_BF16) {  // data gradient of the network's input
                    *reinterpret_cast<__nv_bfloat162 *>(a.out + p * CH + c) = __floats2bfloat162_rn(v0, v1);
                } else {  // EPI_DGELU: data gradient times GELU'(pre-activation below)
                    const __nv_bfloat162 zz = *reinterpret_cast<const __nv_bfloat162 *>(a.aux + p * CH + c);
                    v0 *= gelu_grad(__bfloat162float(zz.x));
                    v1 *= gelu_grad(__bfloat162float(zz.y));
                    *reinterpret_cast<__nv_bfloat162 *>(a.out + p * CH + c) = __floats2bfloat162_rn(v0, v1);
                }
            }
        }
        __syncthreads();  // the slot of plane z-1 is reused by the next prefetch
    }
    cp_wait<0>();
}

// 3x3x3 convolution on tcgen05 (see conv_tc.cuh): same arguments and
// epilogues as k_conv; the input is read through the tensor map `tmap`
// (channels-last [z][y][x][16] BF16, boxes of 8 channels x 130 points x 3 rows).
template <int COUT, int EPI, int CIN, bool BLK = false>
__global__ void __launch_bounds__(convtc::NTHREADS, 2)
    k_conv_tc(const __grid_constant__ CUtensorMap tmap, const ConvArgs a, const convtc::UnitMap um, const int nunits,
              int *err)
{
    using namespace convtc;
    using G = GeoOf<CIN, BLK>;
    extern __shared__ __align__(128) unsigned char sm[];
    uint64_t *full = reinterpret_cast<uint64_t *>(sm);  // [NS] input plane landed
    uint64_t *empty = full + NS;                          // [NS] input plane no longer read
    uint64_t *tfull = empty + NS;                         // [NACC] accumulator set ready
    uint64_t *tempty = tfull + NACC;                      // [NACC] accumulator set read out
    uint64_t *fin = tempty + NACC;                        // all issued MMAs complete
    static_assert((2 * NS + 2 * NACC + 1) * 8 + 8 <= HDR, "barrier header");
    static_assert(RY == 4, "the epilogue reads four rows per accumulator set");
    volatile int *abort_flag = reinterpret_cast<volatile int *>(fin + 1);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(fin + 1) + 1;
    unsigned char *wsm = sm + HDR;
    unsigned char *slots = sm + HDR + G::NTAP * WTAP;
    if (G::SW32)  // swizzled slots start on a 1024-byte boundary
        slots += (1024u - (sa(slots) & 1023u)) & 1023u;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    // weights [tap][co][16 ci] -> [tap t][half][block 0..4: dz = 2, 1, 0, 2, 1][co 0..15][8 ci];
    // rows co >= COUT stay zero.  CIN 16: t = (dy, dx), half = channels 0-7 | 8-15.  CIN 8:
    // t = (dy, pair | single); the pair's halves are dx = -1 | 0, the single's dx = +1 | zero.
    for (int i = threadIdx.x; i < G::NTAP * 2 * WBLK * 16; i += blockDim.x) {
        const int co = i & 15, blk = (i >> 4) % WBLK, half = (i / (16 * WBLK)) & 1, t = i / (32 * WBLK);
        const int dz = (5 - blk) % 3;
        int tap, ci0;
        if (CIN == 16) {
            tap = dz * 9 + t;
            ci0 = half * 8;
        } else {
            tap = (t % 2 == 0) ? dz * 9 + (t / 2) * 3 + half : (half == 0 ? dz * 9 + (t / 2) * 3 + 2 : -1);
            ci0 = 0;
        }
        uint4 v = make_uint4(0, 0, 0, 0);
        if (co < COUT && tap >= 0)
            v = *reinterpret_cast<const uint4 *>(a.wt + (tap * COUT + co) * CH + ci0);
        *reinterpret_cast<uint4 *>(wsm + t * WTAP + half * WHALF + (blk * 16 + co) * 16) = v;
    }
    if (threadIdx.x == 0) {
        for (int s = 0; s < NS; ++s) {
            bar_init(&full[s], 1);
            bar_init(&empty[s], 1);
        }
        for (int b = 0; b < NACC; ++b) {
            bar_init(&tfull[b], 1);
            bar_init(&tempty[b], NEPI);
        }
        bar_init(fin, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // the weight stores (generic proxy) become visible to the tensor cores (async proxy)
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    constexpr int WPROD = NEPI, WMMA = NEPI + 1;
    if (warp == WMMA) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(sa(tmem_slot)),
                     "n"(TCOLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tbase = *tmem_slot;
    if (warp < NEPI) {  // the MMAs only accumulate: every slot starts at zero
        const uint32_t lanes = static_cast<uint32_t>((warp & 3) * 32) << 16;
        for (int c = (warp >> 2) * 8; c < RY * ROWCOLS; c += 16)
            tmem_zero8(tbase + lanes + c);
        tmem_wait_st();
    }
    fence_before();
    __syncthreads();
    fence_after();

    if (warp == WPROD) {
        // ---------------------------------------------------------- producer
        if (lane == 0) {
            int it = 0;
            bool ok = true;
            for (int u = blockIdx.x; u < nunits && ok; u += gridDim.x) {
                int y0, x0, z0, z1;
                um.decode(u, y0, x0, z0, z1);
                for (int p = z0 - 1; p <= z1; ++p) {
                    const int s = it % NS;
                    if (it >= NS && !bar_wait(&empty[s], ((it / NS) - 1) & 1, abort_flag)) {
                        ok = false;
                        break;
                    }
                    bar_expect(&full[s], BOXY * G::ROWB);
                    // blocked view: the box starts at the block of 32 points before x0
                    tma_load_4d(slots + s * G::SLOT, &tmap, &full[s], 0, BLK ? x0 / 32 - 1 : x0 - 1, y0 - 1, p);
                    ++it;
                }
            }
            if (!ok) {
                // let the loads already issued land before the CTA can exit (short bound)
                for (int k = it - NS < 0 ? 0 : it - NS; k < it; ++k) {
                    const unsigned long long t0 = now_ns();
                    while (!bar_try(&full[k % NS], (k / NS) & 1) && now_ns() - t0 < 50000000ull) {
                    }
                }
                atomicCAS(err, 0, static_cast<int>(kDevTimeoutTma));
            }
        }
    } else if (warp == WMMA) {
        // ------------------------------------------------------- MMA issuer
        // (the whole warp runs the loop; elect.sync picks the issuing lane)
        int it = 0, ot = 0;  // input planes consumed, outputs started (over all units)
        bool ok = true;
        const uint32_t wlo = sdesc_lo(sa(wsm), WHALF), slot_lo0 = sdesc_lo(sa(slots), G::LBO_A);
        constexpr uint32_t whi = sdesc_hi(128), ahi = G::SW32 ? sdesc_hi_sw32(256) : sdesc_hi(128);
        for (int u = blockIdx.x; u < nunits && ok; u += gridDim.x) {
            int y0, x0, z0, z1;
            um.decode(u, y0, x0, z0, z1);
            const int nout = z1 - z0;
            // input plane j (z0 - 1 + j) feeds outputs j (dz = 0), j - 1 (dz = 1), j - 2 (dz = 2)
            for (int j = 0; j < nout + 2; ++j, ++it) {
                const int s = it % NS;
                if (!(ok = __all_sync(0xffffffffu, bar_wait(&full[s], (it / NS) & 1, abort_flag))))
                    break;
                fence_after();
                const uint32_t alo = slot_lo0 + static_cast<uint32_t>(s * G::SLOT / 16);
                if (j >= 2 && j < nout) {
                    // all three outputs inside the unit: one N = 48 MMA per tap and row
                    const int o0 = ot + j;  // first taps of output o0: its slot has been read out
                    if (o0 >= NACC) {
                        if (!(ok = __all_sync(0xffffffffu,
                                              bar_wait(&tempty[o0 % NACC], ((o0 / NACC) - 1) & 1, abort_flag))))
                            break;
                        fence_after();
                    }
                    const uint32_t wwin = static_cast<uint32_t>((2 - o0 % NACC) * 256 / 16);
#pragma unroll
                    for (int t = 0; t < G::NTAP; ++t)
#pragma unroll
                        for (int r = 0; r < RY; ++r)
                            mma_bf16_warp(tbase + r * ROWCOLS, alo + G::a_off(t, r) / 16, ahi,
                                          wlo + wwin + t * (WTAP / 16), whi, idesc_bf16(48));
                    mma_commit_warp(&tfull[(o0 - 2) % NACC]);  // output o0 - 2 complete
                } else {
                    // a unit's first or last two planes: one N = 16 MMA per valid output
#pragma unroll
                    for (int dz = 2; dz >= 0; --dz) {
                        const int k = j - dz;  // output index within the unit
                        if (k < 0 || k >= nout)
                            continue;
                        const int o = ot + k, b = o % NACC;
                        if (dz == 0 && o >= NACC) {
                            if (!(ok = __all_sync(0xffffffffu,
                                                  bar_wait(&tempty[b], ((o / NACC) - 1) & 1, abort_flag))))
                                break;
                            fence_after();
                        }
                        const uint32_t wblk = static_cast<uint32_t>((2 - dz) * 256 / 16);
#pragma unroll
                        for (int t = 0; t < G::NTAP; ++t)
#pragma unroll
                            for (int r = 0; r < RY; ++r)
                                mma_bf16_warp(tbase + r * ROWCOLS + b * 16, alo + G::a_off(t, r) / 16, ahi,
                                              wlo + wblk + t * (WTAP / 16), whi, idesc_bf16(16));
                        if (dz == 2)
                            mma_commit_warp(&tfull[b]);  // output o complete
                    }
                    if (!ok)
                        break;
                }
                mma_commit_warp(&empty[s]);  // plane read by all its MMAs
            }
            ot += nout;
        }
        // every issued MMA completes before the tensor memory is released
        mma_commit_warp(fin);
        const unsigned long long t0 = now_ns();
        while (!bar_try(fin, 0) && now_ns() - t0 < 100000000ull) {
        }
        if (!ok && lane == 0)
            atomicCAS(err, 0, static_cast<int>(kDevTimeoutTma));
    } else {
        // ---------------------------------------------------------- epilogue
        const int quad = warp & 3, c0 = (warp >> 2) * 8;  // points 32 quad .., channels c0 .. c0 + 7
        float bias[8];
#pragma unroll
        for (int c = 0; c < 8; ++c)
            bias[c] = (EPI != EPI_DGELU && a.bias && c0 + c < COUT) ? a.bias[c0 + c] : 0.f;
        int ot = 0;
        bool ok = true;
        for (int u = blockIdx.x; u < nunits && ok; u += gridDim.x) {
            int y0, x0, z0, z1;
            um.decode(u, y0, x0, z0, z1);
            const int x = x0 + quad * 32 + lane;
            for (int z = z0; z < z1; ++z) {
                const int b = ot % NACC;
                ok = __all_sync(0xffffffffu, bar_wait(&tfull[b], (ot / NACC) & 1, abort_flag));
                if (!ok)
                    break;
                fence_after();
                float vr[RY][8];
                const uint32_t ta = tbase + (static_cast<uint32_t>(quad * 32) << 16) + b * 16 + c0;
                tmem_ld8x4(ta, ROWCOLS, vr);
#pragma unroll
                for (int r = 0; r < RY; ++r)  // the slot starts the next output at zero
                    tmem_zero8(ta + r * ROWCOLS);
                tmem_wait_st();
                fence_before();
                __syncwarp();
                if (lane == 0)
                    bar_arrive(&tempty[b]);
                ++ot;
                if (x >= a.d.nx || (EPI == EPI_LINEAR_F32 && c0 != 0))
                    continue;
#pragma unroll
                for (int r = 0; r < RY; ++r) {
                const int y = y0 + r;
                if (y >= a.d.ny)
                    break;
                const float (&v)[8] = vr[r];
                const int64_t p = (static_cast<int64_t>(z) * a.d.ny + y) * a.d.nx + x;
                if (EPI == EPI_LINEAR_F32) {
                    a.out_f32[p] = (v[0] + bias[0]) * a.oscale;
                } else if (EPI == EPI_GELU) {
                    // channels >= cout_valid (padding) are zero
                    float2 zv[4];
#pragma unroll
                    for (int c = 0; c < 8; c += 2)
                        zv[c >> 1] = __fadd2_rn(make_float2(v[c], v[c + 1]), make_float2(bias[c], bias[c + 1]));
                    if (c0 + 8 > a.cout_valid) {
#pragma unroll
                        for (int c = 0; c < 8; c += 2) {
                            if (c0 + c >= a.cout_valid)
                                zv[c >> 1].x = 0.f;
                            if (c0 + c + 1 >= a.cout_valid)
                                zv[c >> 1].y = 0.f;
                        }
                    }
                    uint32_t yy[4];
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const float2 g = gelu2(zv[k]);
                        const __nv_bfloat162 yb = __floats2bfloat162_rn(g.x, g.y);
                        yy[k] = *reinterpret_cast<const uint32_t *>(&yb);
                    }
                    *reinterpret_cast<uint4 *>(a.out + p * CH + c0) = make_uint4(yy[0], yy[1], yy[2], yy[3]);
                    if (a.zout) {
                        uint32_t zz[4];
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            const __nv_bfloat162 zb = __floats2bfloat162_rn(zv[k].x, zv[k].y);
                            zz[k] = *reinterpret_cast<const uint32_t *>(&zb);
                        }
                        *reinterpret_cast<uint4 *>(a.zout + p * CH + c0) = make_uint4(zz[0], zz[1], zz[2], zz[3]);
                    }
                } else if (EPI == EPI_LINEAR_BF16) {  // data gradient of the network's input
                    uint32_t oo[4];
#pragma unroll
                    for (int c = 0; c < 8; c += 2) {
                        const __nv_bfloat162 ob = __floats2bfloat162_rn(v[c], v[c + 1]);
                        oo[c >> 1] = *reinterpret_cast<const uint32_t *>(&ob);
                    }
                    *reinterpret_cast<uint4 *>(a.out + p * CH + c0) = make_uint4(oo[0], oo[1], oo[2], oo[3]);
                } else {  // EPI_DGELU: data gradient times GELU'(pre-activation below)
                    const uint4 q0 = *reinterpret_cast<const uint4 *>(a.aux + p * CH + c0);
                    const uint32_t aw[4] = {q0.x, q0.y, q0.z, q0.w};
                    uint32_t oo[4];
#pragma unroll
                    for (int c = 0; c < 8; c += 2) {
                        const __nv_bfloat162 zb = *reinterpret_cast<const __nv_bfloat162 *>(&aw[c >> 1]);
                        const float v0 = v[c] * gelu_grad(__bfloat162float(zb.x));
                        const float v1 = v[c + 1] * gelu_grad(__bfloat162float(zb.y));
                        const __nv_bfloat162 ob = __floats2bfloat162_rn(v0, v1);
                        oo[c >> 1] = *reinterpret_cast<const uint32_t *>(&ob);
                    }
                    *reinterpret_cast<uint4 *>(a.out + p * CH + c0) = make_uint4(oo[0], oo[1], oo[2], oo[3]);
                }
                }
            }
        }
        if (!ok && lane == 0)
            atomicCAS(err, 0, static_cast<int>(kDevTimeoutTma));
    }
    // teardown: the MMA issuer has seen its last MMA complete
    __syncthreads();
    if (warp == WMMA) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "n"(TCOLS) : "memory");
    }
}

// Last layer (16 channels -> 1) on the CUDA cores.  A tensor-core tile would pad
// the single output channel to 16 (the MMA's smallest N); here a CTA owns a
// 64 x 8 (x, y) tile and marches along z, each thread four columns x = x0 + tx +
// 16 j (j = 0..3) of one row.  Every input plane is read once from shared memory
// (the 3 x 3 neighbourhood of each column, 16 channels as 8 pairs) and feeds the
// three output planes it touches -- z+1, z and z-1 -- through three accumulators
// per column, in packed FP32x2 FMAs over channel pairs; each weight pair is read
// once per plane for the four columns.  Output plane z-1 is then complete.  BF16
// weights (the forward layout [tap][8][16], row 0), FP32 accumulation, zero padding.
constexpr int T1X = 64, T1Y = 8, T1NT = 16 * T1Y, H1X = T1X + 2, H1Y = T1Y + 2;
constexpr int P1PTS = H1X * H1Y, P1BYTES = P1PTS * 32, N1SLOT = 3, Z1CH = 16;

__device__ __forceinline__ void load_plane1(unsigned char *slot, const __nv_bfloat16 *in, Dims d, int x0, int y0,
                                            int z)
{
    const bool zin = z >= 0 && z < d.nz;
    for (int idx = threadIdx.x; idx < P1PTS * 2; idx += T1NT) {
        const int pt = idx >> 1, half = idx & 1;
        const int gx = x0 - 1 + pt % H1X, gy = y0 - 1 + pt / H1X;
        const bool valid = zin && gx >= 0 && gx < d.nx && gy >= 0 && gy < d.ny;
        const __nv_bfloat16 *src =
            valid ? in + ((static_cast<int64_t>(z) * d.ny + gy) * d.nx + gx) * CH + half * 8 : in;
        cp_async16(smem_addr(slot + pt * 32 + half * 16), src, valid);
    }
}

__global__ void __launch_bounds__(T1NT) k_conv_out1(const __nv_bfloat16 *in, const __nv_bfloat16 *wt,
                                                     const float *bias, Dims d, float oscale, float *out)
{
    __shared__ float2 w2[27][CH / 2];  // [tap][channel pair]
    extern __shared__ __align__(128) unsigned char ring[];
    const int tiles_x = (d.nx + T1X - 1) / T1X;
    const int x0 = (blockIdx.x % tiles_x) * T1X, y0 = (blockIdx.x / tiles_x) * T1Y;
    const int z0 = blockIdx.y * Z1CH, z1 = min(d.nz, z0 + Z1CH);
    for (int i = threadIdx.x; i < 27 * CH / 2; i += T1NT) {
        const int t = i / (CH / 2), k = i % (CH / 2);
        w2[t][k] = make_float2(__bfloat162float(wt[t * 8 * CH + 2 * k]), __bfloat162float(wt[t * 8 * CH + 2 * k + 1]));
    }
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const int y = y0 + ty;
    const float b = bias ? bias[0] : 0.f;
    const int nin = z1 - z0 + 2;  // input planes z0 - 1 .. z1
    load_plane1(ring, in, d, x0, y0, z0 - 1);
    cp_commit();
    load_plane1(ring + P1BYTES, in, d, x0, y0, z0);
    cp_commit();
    // accumulators of output planes zi - 1 (lo), zi (mid), zi + 1 (hi), per column j (pair sums)
    float2 lo[4], mid[4], hi[4];
#pragma unroll
    for (int j = 0; j < 4; ++j)
        lo[j] = mid[j] = hi[j] = make_float2(0.f, 0.f);
    for (int q = 0; q < nin; ++q) {
        const int zi = z0 - 1 + q;
        if (q + 2 < nin)
            load_plane1(ring + ((q + 2) % N1SLOT) * P1BYTES, in, d, x0, y0, zi + 2);
        cp_commit();
        cp_wait<2>();  // plane q has landed (the two newer groups may be in flight)
        __syncthreads();
        const unsigned char *pl = ring + (q % N1SLOT) * P1BYTES;
#pragma unroll
        for (int dy = 0; dy < 3; ++dy)
#pragma unroll
            for (int dx = 0; dx < 3; ++dx) {
                const int t = dy * 3 + dx;
                uint32_t v[4][8];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const unsigned char *pp = pl + ((ty + dy) * H1X + tx + 16 * j + dx) * 32;
                    const uint4 a = *reinterpret_cast<const uint4 *>(pp);
                    const uint4 c = *reinterpret_cast<const uint4 *>(pp + 16);
                    v[j][0] = a.x, v[j][1] = a.y, v[j][2] = a.z, v[j][3] = a.w;
                    v[j][4] = c.x, v[j][5] = c.y, v[j][6] = c.z, v[j][7] = c.w;
                }
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    // input plane zi reaches output zi + 1 through tap dz = 0, zi through dz = 1,
                    // zi - 1 through dz = 2
                    const float2 wh = w2[t][k], wm = w2[9 + t][k], wl = w2[18 + t][k];
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const float2 x2 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&v[j][k]));
                        hi[j] = __ffma2_rn(wh, x2, hi[j]);
                        mid[j] = __ffma2_rn(wm, x2, mid[j]);
                        lo[j] = __ffma2_rn(wl, x2, lo[j]);
                    }
                }
            }
        __syncthreads();  // the slot of plane q is refilled two iterations later
        if (zi - 1 >= z0 && y < d.ny) {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int x = x0 + tx + 16 * j;
                if (x < d.nx)
                    out[(static_cast<int64_t>(zi - 1) * d.ny + y) * d.nx + x] = ((lo[j].x + lo[j].y) + b) * oscale;
            }
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            lo[j] = mid[j];
            mid[j] = hi[j];
            hi[j] = make_float2(0.f, 0.f);
        }
    }
}

// Last layer (16 channels -> 1) on tcgen05 in tap-split form.  With the output
// o(x, y, z) = sum over (dz, dy, dx, ci) of W[dz][dy][dx][ci] h(x+dx-1, y+dy-1, z+dz-1)[ci],
// the tensor cores first contract the channels and the x taps of every input row:
//   Y_n(x, y', p) = sum over (dx, ci) of W[dz][dy][dx][ci] h(x+dx-1, y', p)[ci],  n = 3 dz + dy,
// three N = 16 MMAs (dx = 0, 1, 2: the plane slot shifted by dx points; columns
// n = 0..8 used) per input row and plane, into tensor memory; the CUDA cores then
// add the nine (dy, dz) terms: o(x, y, z) = sum over (dz, dy) of Y_{3dz+dy}(x, y+dy-1, z+dz-1).
// Per plane a CTA (128 x-points, RY = 4 output rows) issues 6 x 3 MMAs for its 6
// input rows, against 9 N = 48 MMAs per output row in the general kernel: a third
// of the A-tile reads from shared memory.  The producer warp and the plane ring are
// the general kernel's; each plane is one 32-byte swizzled box (out1tc::BOXX).
// Epilogue warp w reads lanes 32 (w & 3) .. +31 (points) and output rows 2 (w >> 2)
// and 2 (w >> 2) + 1, i.e. input rows 2 (w >> 2) .. +3 of each plane; each plane
// feeds output planes p + 1 (dz = 0), p (dz = 1) and p - 1 (dz = 2), kept in three
// rotating registers per row; output p - 1 is then complete.  The terms of an
// output add in a fixed order: planes in z order, within a plane dy = 0, 1, 2.
namespace out1tc {
constexpr int NSET = 2;                  // accumulator sets (one input plane each)
constexpr int SETCOLS = 6 * 16;          // 6 input rows x 16 columns
constexpr int TCOLS = 256;               // allocated tensor-memory columns
constexpr int WDX = 2 * 16 * 16;         // bytes of one dx weight matrix: [half][16 rows][8 ci] BF16
constexpr int NSLOT = 4;                 // plane slots
// Input planes: one TMA box of all 16 channels per plane (32-byte rows, the 32-byte
// swizzled K-major layout), rows of 136 points so that every row starts on a 256-byte
// pattern boundary; two boxes of 8 channels (16-byte rows, each half of an L2 sector)
// made twice the L2 requests, which bounded the kernel.
constexpr int BOXX = 136;
constexpr int ROWB = BOXX * 32;
constexpr int SLOT = (convtc::BOXY * ROWB + 1023) / 1024 * 1024;
constexpr int SMEM = convtc::HDR + 3 * WDX + 1024 + NSLOT * SLOT;
}  // namespace out1tc

// D[tmem] (+)= A B as mma_bf16_warp, with the accumulate flag a runtime value.
__device__ __forceinline__ void mma_bf16_warp_acc(uint32_t d_tmem, uint32_t alo, uint32_t ahi, uint32_t blo,
                                                  uint32_t bhi, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred e, a;\n\t.reg .b32 l;\n\t.reg .b64 da, db;\n\t"
        "setp.ne.b32 a, %6, 0;\n\t"
        "elect.sync l|e, 0xffffffff;\n\t"
        "mov.b64 da, {%1, %2};\n\t"
        "mov.b64 db, {%3, %4};\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], da, db, %5, a;\n\t}" ::"r"(d_tmem),
        "r"(alo), "r"(ahi), "r"(blo), "r"(bhi), "r"(idesc), "r"(acc));
}

// Columns 0..8 of one tensor-memory row set for the warp's 32 lanes (no wait).
__device__ __forceinline__ void tmem_ld9(uint32_t taddr, uint32_t (&r)[9])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];" : "=r"(r[8]) : "r"(taddr + 8));
}

__global__ void __launch_bounds__(convtc::NTHREADS, 2)
    k_conv_out1_tc(const __grid_constant__ CUtensorMap tmap, const ConvArgs a, const convtc::UnitMap um,
                   const int nunits, int *err)
{
    using namespace convtc;
    using out1tc::NSET;
    using out1tc::NSLOT;
    using out1tc::SETCOLS;
    using out1tc::WDX;
    extern __shared__ __align__(128) unsigned char sm[];
    uint64_t *full = reinterpret_cast<uint64_t *>(sm);  // [NSLOT] input plane landed
    uint64_t *empty = full + NSLOT;                       // [NSLOT] input plane no longer read
    uint64_t *tfull = empty + NSLOT;                      // [NSET] accumulator set ready
    uint64_t *tempty = tfull + NSET;                      // [NSET] accumulator set read out
    uint64_t *fin = tempty + NSET;                        // all issued MMAs complete
    static_assert((2 * NSLOT + 2 * NSET + 1) * 8 + 8 <= HDR, "barrier header");
    static_assert(RY == 4 && BOXY == 6, "six input rows per plane for four output rows");
    volatile int *abort_flag = reinterpret_cast<volatile int *>(fin + 1);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(fin + 1) + 1;
    unsigned char *wsm = sm + HDR;
    unsigned char *slots = sm + HDR + 3 * WDX;
    slots += (1024u - (sa(slots) & 1023u)) & 1023u;  // swizzled slots start on a 1024-byte boundary
    constexpr int SLOTB = out1tc::SLOT;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    // weights [tap][8][16] (row 0 real) -> [dx][half][n = 3 dz + dy][8 ci]; rows n >= 9 zero
    for (int i = threadIdx.x; i < 3 * 2 * 16; i += blockDim.x) {
        const int n = i & 15, half = (i >> 4) & 1, dx = i >> 5;
        uint4 v = make_uint4(0, 0, 0, 0);
        if (n < 9) {
            const int dz = n / 3, dy = n % 3;
            v = *reinterpret_cast<const uint4 *>(a.wt + (((dz * 3 + dy) * 3 + dx) * 8) * CH + half * 8);
        }
        *reinterpret_cast<uint4 *>(wsm + dx * WDX + half * 256 + n * 16) = v;
    }
    if (threadIdx.x == 0) {
        for (int s = 0; s < NSLOT; ++s) {
            bar_init(&full[s], 1);
            bar_init(&empty[s], 1);
        }
        for (int b = 0; b < NSET; ++b) {
            bar_init(&tfull[b], 1);
            bar_init(&tempty[b], NEPI);
        }
        bar_init(fin, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    constexpr int WPROD = NEPI, WMMA = NEPI + 1;
    if (warp == WMMA) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(sa(tmem_slot)),
                     "n"(out1tc::TCOLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tbase = *tmem_slot;

    if (warp == WPROD) {
        // ---------------------------------------------------------- producer
        if (lane == 0) {
            int it = 0;
            bool ok = true;
            for (int u = blockIdx.x; u < nunits && ok; u += gridDim.x) {
                int y0, x0, z0, z1;
                um.decode(u, y0, x0, z0, z1);
                for (int p = z0 - 1; p <= z1; ++p) {
                    const int s = it % NSLOT;
                    if (it >= NSLOT && !bar_wait(&empty[s], ((it / NSLOT) - 1) & 1, abort_flag)) {
                        ok = false;
                        break;
                    }
                    bar_expect(&full[s], BOXY * out1tc::ROWB);
                    tma_load_4d(slots + s * SLOTB, &tmap, &full[s], 0, x0 - 1, y0 - 1, p);
                    ++it;
                }
            }
            if (!ok) {
                for (int k = it - NSLOT < 0 ? 0 : it - NSLOT; k < it; ++k) {
                    const unsigned long long t0 = now_ns();
                    while (!bar_try(&full[k % NSLOT], (k / NSLOT) & 1) && now_ns() - t0 < 50000000ull) {
                    }
                }
                atomicCAS(err, 0, static_cast<int>(kDevTimeoutTma));
            }
        }
    } else if (warp == WMMA) {
        // ------------------------------------------------------- MMA issuer
        int it = 0;  // input planes over all units (plane it uses slot it % NSLOT and set it % NSET)
        bool ok = true;
        const uint32_t wlo = sdesc_lo(sa(wsm), 256);
        constexpr uint32_t whi = sdesc_hi(128);
        for (int u = blockIdx.x; u < nunits && ok; u += gridDim.x) {
            int y0, x0, z0, z1;
            um.decode(u, y0, x0, z0, z1);
            for (int p = z0 - 1; p <= z1; ++p, ++it) {
                const int s = it % NSLOT, b = it % NSET;
                if (!(ok = __all_sync(0xffffffffu, bar_wait(&full[s], (it / NSLOT) & 1, abort_flag))))
                    break;
                if (it >= NSET &&
                    !(ok = __all_sync(0xffffffffu, bar_wait(&tempty[b], ((it / NSET) - 1) & 1, abort_flag))))
                    break;
                fence_after();
                // K-major, 32-byte swizzle: rows of 32 bytes (16 channels), 8-row groups
                // 256 bytes apart; the x tap dx starts the operand dx rows later (the
                // swizzle is a function of the shared-memory address, as the TMA wrote it)
                const uint32_t sbase = sa(slots + s * SLOTB);
#pragma unroll
                for (int r = 0; r < BOXY; ++r)
#pragma unroll
                    for (int dx = 0; dx < 3; ++dx)
                        mma_bf16_warp_acc(tbase + b * SETCOLS + r * 16,
                                          sdesc_lo(sbase + static_cast<uint32_t>(r * out1tc::ROWB + dx * 32), 16),
                                          sdesc_hi_sw32(256), wlo + static_cast<uint32_t>(dx * WDX / 16), whi,
                                          idesc_bf16(16), dx > 0 ? 1u : 0u);
                mma_commit_warp(&tfull[b]);   // the set of plane it is complete
                mma_commit_warp(&empty[s]);   // plane read by all its MMAs
            }
        }
        mma_commit_warp(fin);
        const unsigned long long t0 = now_ns();
        while (!bar_try(fin, 0) && now_ns() - t0 < 100000000ull) {
        }
        if (!ok && lane == 0)
            atomicCAS(err, 0, static_cast<int>(kDevTimeoutTma));
    } else {
        // ---------------------------------------------------------- epilogue
        const int quad = warp & 3, h = warp >> 2;  // points 32 quad .., output rows 2h, 2h + 1
        const float bias = a.bias ? a.bias[0] : 0.f;
        int it = 0;
        bool ok = true;
        for (int u = blockIdx.x; u < nunits && ok; u += gridDim.x) {
            int y0, x0, z0, z1;
            um.decode(u, y0, x0, z0, z1);
            const int x = x0 + quad * 32 + lane;
            // output planes p - 1 (lo), p (mid), p + 1 (hi) of rows 2h + j
            float lo[2] = {0.f, 0.f}, mid[2] = {0.f, 0.f}, hi[2] = {0.f, 0.f};
            for (int p = z0 - 1; p <= z1; ++p, ++it) {
                const int b = it % NSET;
                ok = __all_sync(0xffffffffu, bar_wait(&tfull[b], (it / NSET) & 1, abort_flag));
                if (!ok)
                    break;
                fence_after();
                uint32_t rv[4][9];
                const uint32_t ta = tbase + (static_cast<uint32_t>(quad * 32) << 16) + b * SETCOLS + 2 * h * 16;
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    tmem_ld9(ta + i * 16, rv[i]);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    asm volatile(""
                                 : "+r"(rv[i][0]), "+r"(rv[i][1]), "+r"(rv[i][2]), "+r"(rv[i][3]), "+r"(rv[i][4]),
                                   "+r"(rv[i][5]), "+r"(rv[i][6]), "+r"(rv[i][7]), "+r"(rv[i][8]));
                fence_before();
                __syncwarp();
                if (lane == 0)
                    bar_arrive(&tempty[b]);
                // plane p reaches output p + 1 - dz through dz; row 2h + j reads input rows 2h + j + dy
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    float c[3];
#pragma unroll
                    for (int dz = 0; dz < 3; ++dz)
                        c[dz] = (__uint_as_float(rv[j][3 * dz]) + __uint_as_float(rv[j + 1][3 * dz + 1])) +
                                __uint_as_float(rv[j + 2][3 * dz + 2]);
                    hi[j] += c[0];
                    mid[j] += c[1];
                    lo[j] += c[2];
                }
                const int zo = p - 1;  // complete: it has had planes zo - 1, zo and zo + 1
                if (zo >= z0 && x < a.d.nx) {
#pragma unroll
                    for (int j = 0; j < 2; ++j) {
                        const int y = y0 + 2 * h + j;
                        if (y < a.d.ny)
                            a.out_f32[(static_cast<int64_t>(zo) * a.d.ny + y) * a.d.nx + x] = (lo[j] + bias) * a.oscale;
                    }
                }
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    lo[j] = mid[j];
                    mid[j] = hi[j];
                    hi[j] = 0.f;
                }
            }
        }
        if (!ok && lane == 0)
            atomicCAS(err, 0, static_cast<int>(kDevTimeoutTma));
    }
    __syncthreads();
    if (warp == WMMA) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "n"(out1tc::TCOLS)
                     : "memory");
    }
}

struct WgradArgs {
    const __nv_bfloat16 *x;   // layer input [z][y][x][16]
    const __nv_bfloat16 *dz;  // output gradient [z][y][x][16]
    float *grad_w;            // master-order gradient of this layer's weights [co][ci][27]
    float *grad_b;            // [co]
    Dims d;
    int cin, cout;            // real channel counts
};

// dW[co][ci][tap] += sum_p x[p + tap][ci] dz[p][co];  db[co] += sum_p dz[p][co].
// Warp w owns taps w, w+8, w+16, w+24; per 16-point chunk the tensor cores
// compute a (ci x points) x (points x co) product.
__global__ void __launch_bounds__(NTHR) k_wgrad(const WgradArgs a)
{
    extern __shared__ __align__(128) unsigned char sm[];
    unsigned char *ring = sm;                              // NSLOT halo planes of x
    unsigned char *dzs = sm + NSLOT * PLANE_BYTES;         // 2 slots of the dz tile
    constexpr int DZ_BYTES = TXC * TYC * 32;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int tiles_x = (a.d.nx + TXC - 1) / TXC;
    const int x0 = (blockIdx.x % tiles_x) * TXC, y0 = (blockIdx.x / tiles_x) * TYC;
    const int z0 = blockIdx.y * ZCHUNK;
    const int z1 = min(a.d.nz, z0 + ZCHUNK);
    const int m = lane >> 3, r = lane & 7;
    const int g = lane >> 2, q = lane & 3;

    float acc[4][2][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int t = 0; t < 2; ++t)
#pragma unroll
            for (int k = 0; k < 4; ++k)
                acc[i][t][k] = 0.f;
    float bsum = 0.f;  // thread tid < 16: db of channel tid over this CTA

    load_plane(ring + 0 * PLANE_BYTES, a.x, a.d, x0, y0, z0 - 1);
    load_plane(ring + 1 * PLANE_BYTES, a.x, a.d, x0, y0, z0);
    cp_commit();
    for (int z = z0; z < z1; ++z) {
        load_plane(ring + ((z + 1 - z0 + 1) % NSLOT) * PLANE_BYTES, a.x, a.d, x0, y0, z + 1);
        load_tile(dzs + (z & 1) * DZ_BYTES, a.dz, a.d, x0, y0, z);
        cp_commit();
        cp_wait<0>();
        __syncthreads();
        const unsigned char *dzt = dzs + (z & 1) * DZ_BYTES;
        if (tid < 16) {
            for (int pt = 0; pt < TXC * TYC; ++pt) {
                const __nv_bfloat16 *row = reinterpret_cast<const __nv_bfloat16 *>(dzt + swz(pt, tid >> 3));
                bsum += __bfloat162float(row[tid & 7]);
            }
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int tap = warp + 8 * i;
            if (tap >= 27)
                break;
            const int kz = tap / 9, ky = (tap / 3) % 3, kx = tap % 3;
            const unsigned char *slot = ring + ((z + kz - 1 - z0 + 1) % NSLOT) * PLANE_BYTES;
#pragma unroll
            for (int chunk = 0; chunk < TYC * 2; ++chunk) {
                const int cy = chunk >> 1, cs = chunk & 1;
                // A = x^T (ci x 16 points): matrices (ci 0-7|8-15) x (points 0-7|8-15), transposed loads
                const int apt = (cy + ky) * HX + cs * 16 + r + 8 * (m >> 1) + kx;
                uint32_t a0, a1, a2, a3;
                ldsm_x4_t(smem_addr(slot + swz(apt, m & 1)), a0, a1, a2, a3);
                // B = dz (16 points x co) column-major fragments for the two 8-channel tiles
                const int bpt = cy * TXC + cs * 16 + r + 8 * (m & 1);
                uint32_t b0, b1, b2, b3;
                ldsm_x4_t(smem_addr(dzt + swz(bpt, m >> 1)), b0, b1, b2, b3);
                mma16816(acc[i][0], a0, a1, a2, a3, b0, b1);
                mma16816(acc[i][1], a0, a1, a2, a3, b2, b3);
            }
        }
        __syncthreads();
    }
    // C rows = ci (g, g+8), cols = co (8t + 2q, +1)
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int tap = warp + 8 * i;
        if (tap >= 27)
            break;
#pragma unroll
        for (int t = 0; t < 2; ++t)
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int ci = g + 8 * (k >> 1), co = 8 * t + 2 * q + (k & 1);
                if (ci < a.cin && co < a.cout)
                    atomicAdd(&a.grad_w[(co * a.cin + ci) * 27 + tap], acc[i][t][k]);
            }
    }
    if (tid < 16 && tid < a.cout)
        atomicAdd(&a.grad_b[tid], bsum);
}

// x = s (u+, u^n, c_norm^2 u+, c_norm^2 u^n, 0...) channels-last BF16: every
// channel vanishes with the field, so with zero biases a zero field gets a zero
// correction.
__global__ void k_prep(const float *up, const float *un, const float *cn, float s, int64_t n, __nv_bfloat16 *x)
{
    for (int64_t p = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; p < n;
         p += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        __nv_bfloat162 *o = reinterpret_cast<__nv_bfloat162 *>(x + p * CH);
        const float a = s * up[p], b = s * un[p], c2 = cn[p] * cn[p];
        o[0] = __floats2bfloat162_rn(a, b);
        o[1] = __floats2bfloat162_rn(c2 * a, c2 * b);
#pragma unroll
        for (int k = 2; k < 8; ++k)
            o[k] = __floats2bfloat162_rn(0.f, 0.f);
    }
}

// loss += sum (o - s (ref - u+))^2;  dOut = 2 (o - target) / n into channel 0 of a 16-channel tensor.
__global__ void k_loss(const float *o, const float *up, const float *ref, float s, float wgt, int64_t n,
                       double *loss, __nv_bfloat16 *dout)
{
    double acc = 0.0;
    for (int64_t p = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; p < n;
         p += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const float d = o[p] - s * (ref[p] - up[p]);  // s: the output scale
        acc += static_cast<double>(d) * d;
        __nv_bfloat162 *g = reinterpret_cast<__nv_bfloat162 *>(dout + p * CH);
        g[0] = __floats2bfloat162_rn(2.0f * wgt * d / static_cast<float>(n), 0.f);
#pragma unroll
        for (int k = 1; k < 8; ++k)
            g[k] = __floats2bfloat162_rn(0.f, 0.f);
    }
    for (int off = 16; off > 0; off >>= 1)
        acc += __shfl_down_sync(0xffffffffu, acc, off);
    if ((threadIdx.x & 31) == 0)
        atomicAdd(loss, acc);
}

// Master FP32 weights -> BF16 forward [tap][co_pad][16] and data-gradient [tap'][ci][16] layouts.
__global__ void k_convert(const float *w, int cin, int cout, int cout_pad, __nv_bfloat16 *fwd, __nv_bfloat16 *bwd)
{
    const int n = 27 * CH * CH;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int tap = i / (CH * CH), a = (i / CH) % CH, b = i % CH;
        // forward: row (tap, co = a), column ci = b
        if (a < cout_pad)
            fwd[(tap * cout_pad + a) * CH + b] =
                __float2bfloat16_rn((a < cout && b < cin) ? w[(a * cin + b) * 27 + tap] : 0.f);
        // data gradient: output channel ci = a, input channel co = b, tap flipped
        if (bwd)
            bwd[(tap * CH + a) * CH + b] =
                __float2bfloat16_rn((a < cin && b < cout) ? w[(b * cin + a) * 27 + (26 - tap)] : 0.f);
    }
}

// (1 - beta) is passed in: 1 - 0.999f evaluated in FP32 is off by 1.3e-5.
struct BiasRanges {
    int lo[3], hi[3];  // [lo, hi) index ranges of the three bias vectors; empty when not frozen
};

__global__ void k_adam(float *p, const float *g, float *m1, float *m2, int n, float lr, float b1, float b2,
                       float omb1, float omb2, float eps, float bc1, float bc2, BiasRanges frozen,
                       const unsigned char *trainable)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        if ((i >= frozen.lo[0] && i < frozen.hi[0]) || (i >= frozen.lo[1] && i < frozen.hi[1]) ||
            (i >= frozen.lo[2] && i < frozen.hi[2]) || (trainable && !trainable[i]))
            continue;
        const float gi = g[i];
        const float mi = b1 * m1[i] + omb1 * gi;
        const float vi = b2 * m2[i] + omb2 * gi * gi;
        m1[i] = mi;
        m2[i] = vi;
        p[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
    }
}

// dout channel 0 = g / t (the correction is o / t), the other channels 0.
__global__ void k_seed(const float *g, float inv_t, int64_t n, __nv_bfloat16 *dout)
{
    for (int64_t p = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; p < n;
         p += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        __nv_bfloat162 *q = reinterpret_cast<__nv_bfloat162 *>(dout + p * CH);
        q[0] = __floats2bfloat162_rn(g[p] * inv_t, 0.f);
#pragma unroll
        for (int k = 1; k < 8; ++k)
            q[k] = __floats2bfloat162_rn(0.f, 0.f);
    }
}

__global__ void k_gelu(const float *x, float *y, int64_t n)
{
    for (int64_t p = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; p < n;
         p += static_cast<int64_t>(gridDim.x) * blockDim.x)
        y[p] = gelu(x[p]);
}

__global__ void k_scale_add(float *dst, const float *src, float scale, int64_t n)
{
    for (int64_t p = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; p < n;
         p += static_cast<int64_t>(gridDim.x) * blockDim.x)
        dst[p] += scale * src[p];
}

}  // namespace
}  // namespace gbst

// ===========================================================================
using namespace gbst;

struct gbst_closure_s {
    int cin = 3, hidden = 16;
    int64_t max_pts = 0;
    double scale = 1.0;
    cudaStream_t stream = nullptr;
    gbst_allocator alloc{};
    bool custom = false;
    std::vector<std::pair<void *, size_t>> owned;
    // parameters (master FP32, oracle order) and their offsets
    int64_t off[6] = {0}, cnt[6] = {0}, nparams = 0;
    float *p = nullptr, *g = nullptr, *m1 = nullptr, *m2 = nullptr;
    int64_t t = 0;  // Adam step
    __nv_bfloat16 *wf[3] = {nullptr}, *wb[3] = {nullptr};
    // activations
    __nv_bfloat16 *x = nullptr, *z1 = nullptr, *y1 = nullptr, *z2 = nullptr, *y2 = nullptr;
    __nv_bfloat16 *dout = nullptr, *dz2 = nullptr, *dz1 = nullptr;
    float *o = nullptr;
    double *dloss = nullptr;
    bool weights_dirty = true;
    double out_scale = 1.0;     // target in network units: out_scale * (u_ref - u+)
    bool freeze_biases = false; // Adam leaves the biases unchanged
    double loss_weight = 1.0;   // factor on the loss (and its gradient) of the next loss_grad calls
    int conv_impl = 0;          // 0: tcgen05 (last layer tap-split), 1: mma.sync, 2: tcgen05 with the last
                                // layer on the CUDA cores, 3: tcgen05 with the last layer as the hidden ones
    int *derr = nullptr;        // device error word of the tcgen05 convolutions
    unsigned char *trainable = nullptr;      // per-parameter Adam mask (null: all parameters train)
    unsigned char *trainable_buf = nullptr;  // its device storage
    bool layer_grad[3] = {true, true, true}; // layer l has a trainable weight or bias: its dW, db are computed
    // feature inputs (cin 8): FP32 stencil features, see closure_set_features
    bool feat = false;
    int feat_r = 2;
    double feat_w[5] = {0, 0, 0, 0, 0};
    double feat_s[8] = {1, 1, 1, 1, 1, 1, 1, 1};
    ClosureFeatBufs fb;
    __nv_bfloat16 *dx = nullptr;  // cotangent of the network input (backward to the fields)
};

cudaStream_t gbst::closure_stream(gbst_closure c) { return c ? c->stream : nullptr; }
bool gbst::closure_has_features(gbst_closure c) { return c && c->feat; }

namespace {

void *cl_alloc(gbst_closure c, size_t bytes)
{
    void *ptr = nullptr;
    if (c->custom)
        ptr = c->alloc.alloc(bytes, c->stream, c->alloc.ctx);
    else if (cudaMalloc(&ptr, bytes) != cudaSuccess) {
        cudaGetLastError();
        ptr = nullptr;
    }
    if (ptr)
        c->owned.emplace_back(ptr, bytes);
    return ptr;
}

int blocks_for(int64_t n) { return static_cast<int>(std::min<int64_t>(8192, (n + 255) / 256)); }

size_t conv_smem(int cout) { return 27 * cout * 32 + NSLOT * PLANE_BYTES; }
size_t wgrad_smem() { return NSLOT * PLANE_BYTES + 2 * TXC * TYC * 32; }

template <int COUT, int EPI>
cudaError_t launch_conv(const ConvArgs &a, cudaStream_t s)
{
    const size_t smem = conv_smem(COUT);
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(reinterpret_cast<const void *>(&k_conv<COUT, EPI>),
                             cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
        attr = true;
    }
    const int tiles = ((a.d.nx + TXC - 1) / TXC) * ((a.d.ny + TYC - 1) / TYC);
    dim3 grid(tiles, (a.d.nz + ZCHUNK - 1) / ZCHUNK);
    k_conv<COUT, EPI><<<grid, NTHR, smem, s>>>(a);
    return cudaGetLastError();
}

int num_sms_dev()
{
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
}

// CIN: channels per point of the input (16, or 8 for the packed feature input of layer 1).
template <int COUT, int EPI, int CIN = 16, bool BLK = false>
cudaError_t launch_conv_tc(const ConvArgs &a, int *err, cudaStream_t s)
{
    using namespace convtc;
    using G = GeoOf<CIN, BLK>;
    constexpr int smem = tc_smem<CIN, BLK>();
    static int occ = -1;
    if (occ < 0) {
        const void *fn = reinterpret_cast<const void *>(&k_conv_tc<COUT, EPI, CIN, BLK>);
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        // the largest shared-memory carveout, so that two CTAs fit on an SM
        cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, NTHREADS, smem) != cudaSuccess || occ < 1) {
            cudaGetLastError();
            occ = 2;
        }
        // (the query answered 1 on GB300 although the launch's limits from registers and shared
        // memory are both 2; a grid of two CTAs per SM runs as one wave when both fit and as two
        // otherwise, as the units are strided over the grid).  Tensor memory (256 columns per
        // CTA) allows no more than two.
        occ = 2;
    }
    // activation [z][y][x][CIN] BF16: dims (channel, x, y, z), boxes of CIN channels x BOXX points x 6
    // rows; blocked view (BLK, nx a multiple of 32): dims (32 points x 8 channels, x / 32, y, z),
    // boxes of 6 blocks x 6 rows
    CUtensorMap m;
    const uint64_t row_bytes = static_cast<uint64_t>(a.d.nx) * CIN * 2;
    if (BLK && a.d.nx % 32 != 0)
        return cudaErrorInvalidValue;
    const uint64_t dims[4] = {BLK ? 256ull : static_cast<uint64_t>(CIN),
                              static_cast<uint64_t>(BLK ? a.d.nx / 32 : a.d.nx), static_cast<uint64_t>(a.d.ny),
                              static_cast<uint64_t>(a.d.nz)};
    const uint64_t strides[3] = {BLK ? 512ull : CIN * 2ull, row_bytes, row_bytes * a.d.ny};
    const uint32_t box[4] = {BLK ? 256u : static_cast<uint32_t>(CIN),
                             static_cast<uint32_t>(BLK ? GeoB8::BLOCKS : G::BOXX), BOXY, 1};
    std::string msg;
    if (!encode_tmap_bf16_4d(&m, a.in, dims, strides, box, &msg, G::SW32))
        return cudaErrorInvalidValue;
    UnitMap um{(a.d.nx + TXP - 1) / TXP, (a.d.nz + ZCH - 1) / ZCH, (a.d.ny + RY - 1) / RY, a.d.nz};
    const int64_t nunits = static_cast<int64_t>(um.nxc) * um.nyc * um.nzc;
    if (nunits > (1ll << 31) - 1)
        return cudaErrorInvalidValue;
    const int ctas = static_cast<int>(std::min<int64_t>(nunits, static_cast<int64_t>(num_sms_dev()) * occ));
    k_conv_tc<COUT, EPI, CIN, BLK><<<ctas, NTHREADS, smem, s>>>(m, a, um, static_cast<int>(nunits), err);
    return cudaGetLastError();
}

// The one-channel last layer in tap-split form on tcgen05 (k_conv_out1_tc): the
// general kernel's input staging and work units, two CTAs per SM.
cudaError_t launch_conv_out1_tc(const ConvArgs &a, int *err, cudaStream_t s)
{
    using namespace convtc;
    constexpr int smem = out1tc::SMEM;
    static bool attr = false;
    if (!attr) {
        const void *fn = reinterpret_cast<const void *>(&k_conv_out1_tc);
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        attr = true;
    }
    CUtensorMap m;
    const uint64_t dims[4] = {16ull, static_cast<uint64_t>(a.d.nx), static_cast<uint64_t>(a.d.ny),
                              static_cast<uint64_t>(a.d.nz)};
    const uint64_t strides[3] = {32ull, static_cast<uint64_t>(a.d.nx) * 32, static_cast<uint64_t>(a.d.nx) * a.d.ny * 32};
    const uint32_t box[4] = {16u, static_cast<uint32_t>(out1tc::BOXX), BOXY, 1};
    std::string msg;
    if (!encode_tmap_bf16_4d(&m, a.in, dims, strides, box, &msg, true))
        return cudaErrorInvalidValue;
    UnitMap um{(a.d.nx + TXP - 1) / TXP, (a.d.nz + ZCH - 1) / ZCH, (a.d.ny + RY - 1) / RY, a.d.nz};
    const int64_t nunits = static_cast<int64_t>(um.nxc) * um.nyc * um.nzc;
    if (nunits > (1ll << 31) - 1)
        return cudaErrorInvalidValue;
    // two CTAs per SM (tensor memory: 256 columns each)
    const int ctas = static_cast<int>(std::min<int64_t>(nunits, static_cast<int64_t>(num_sms_dev()) * 2));
    k_conv_out1_tc<<<ctas, NTHREADS, smem, s>>>(m, a, um, static_cast<int>(nunits), err);
    return cudaGetLastError();
}

// The convolution of the closure's selected implementation.
template <int COUT, int EPI>
cudaError_t conv(gbst_closure c, const ConvArgs &a)
{
    return c->conv_impl != 1 ? launch_conv_tc<COUT, EPI>(a, c->derr, c->stream) : launch_conv<COUT, EPI>(a, c->stream);
}

// Device error word of the tcgen05 kernels (a bounded wait expired): reported once, then cleared.
gbst_status check_device_error(gbst_closure c)
{
    int code = 0;
    cudaError_t e = cudaMemcpyAsync(&code, c->derr, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess)
        return record_error(GBST_ECUDA, cudaGetErrorString(e));
    if (code != 0) {
        cudaMemsetAsync(c->derr, 0, sizeof(int), c->stream);
        return record_error(GBST_ETIMEOUT, "closure: a bounded device-side wait expired");
    }
    return GBST_OK;
}

cudaError_t launch_wgrad(const WgradArgs &a, cudaStream_t s)
{
    const size_t smem = wgrad_smem();
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(reinterpret_cast<const void *>(&k_wgrad), cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(smem));
        attr = true;
    }
    const int tiles = ((a.d.nx + TXC - 1) / TXC) * ((a.d.ny + TYC - 1) / TYC);
    dim3 grid(tiles, (a.d.nz + ZCHUNK - 1) / ZCHUNK);
    k_wgrad<<<grid, NTHR, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_conv_out1(const ConvArgs &a, cudaStream_t s)
{
    static bool attr = false;
    const int smem = N1SLOT * P1BYTES;
    if (!attr) {
        cudaFuncSetAttribute(reinterpret_cast<const void *>(&k_conv_out1), cudaFuncAttributeMaxDynamicSharedMemorySize,
                             smem);
        attr = true;
    }
    const int tiles = ((a.d.nx + T1X - 1) / T1X) * ((a.d.ny + T1Y - 1) / T1Y);
    dim3 grid(tiles, (a.d.nz + Z1CH - 1) / Z1CH);
    k_conv_out1<<<grid, T1NT, smem, s>>>(a.in, a.wt, a.bias, a.d, a.oscale, a.out_f32);
    return cudaGetLastError();
}

gbst_status check_dims(gbst_closure c, int64_t nx, int64_t ny, int64_t nz, Dims *d)
{
    if (nx < 1 || ny < 1 || nz < 1 || nx * ny * nz > c->max_pts || nx > (1 << 30) || ny > (1 << 30) ||
        nz > (1 << 30))
        return record_error(GBST_EINVAL, "closure: grid larger than the size given at closure_create");
    d->nx = static_cast<int>(nx);
    d->ny = static_cast<int>(ny);
    d->nz = static_cast<int>(nz);
    return GBST_OK;
}

gbst_status refresh_weights(gbst_closure c)
{
    if (!c->weights_dirty)
        return GBST_OK;
    const int cins[3] = {c->cin, c->hidden, c->hidden}, couts[3] = {c->hidden, c->hidden, 1};
    const int pads[3] = {CH, CH, 8};
    for (int l = 0; l < 3; ++l) {
        k_convert<<<8, 256, 0, c->stream>>>(c->p + c->off[2 * l], cins[l], couts[l], pads[l], c->wf[l], c->wb[l]);
    }
    c->weights_dirty = false;
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? GBST_OK : record_error(GBST_ECUDA, cudaGetErrorString(e));
}

// Forward pass into out (default c->o, network units) times oscale.  keep: also store the
// pre-activations.
gbst_status forward(gbst_closure c, const float *up, const float *un, const float *cn, Dims d, bool keep,
                    float *out = nullptr, float oscale = 1.0f)
{
    gbst_status st = refresh_weights(c);
    if (st != GBST_OK)
        return st;
    const int64_t n = static_cast<int64_t>(d.nx) * d.ny * d.nz;
    // inference on the tensor cores: the 8 feature channels packed at 16 bytes per point, layer 1
    // with K = 16 spanning a point and its x neighbour
    const bool x8 = c->feat && !keep && c->conv_impl != 1;
    if (c->feat) {
        st = closure_features_forward(up, un, cn, d.nx, d.ny, d.nz, c->feat_r, c->feat_w, c->feat_s, c->fb, c->x,
                                      keep, x8 ? 8 : 16, c->stream);
        if (st != GBST_OK)
            return st;
    } else {
        k_prep<<<blocks_for(n), 256, 0, c->stream>>>(up, un, cn, static_cast<float>(c->scale), n, c->x);
    }
    ConvArgs a{};
    a.d = d;
    a.in = c->x;
    a.wt = c->wf[0];
    a.bias = c->p + c->off[1];
    a.out = c->y1;
    a.zout = keep ? c->z1 : nullptr;
    a.cout_valid = c->hidden;
    cudaError_t e = !x8              ? conv<16, EPI_GELU>(c, a)
                    : d.nx % 32 == 0 ? launch_conv_tc<16, EPI_GELU, 8, true>(a, c->derr, c->stream)
                                     : launch_conv_tc<16, EPI_GELU, 8>(a, c->derr, c->stream);
    a.in = c->y1;
    a.wt = c->wf[1];
    a.bias = c->p + c->off[3];
    a.out = c->y2;
    a.zout = keep ? c->z2 : nullptr;
    if (e == cudaSuccess)
        e = conv<16, EPI_GELU>(c, a);
    ConvArgs b{};
    b.d = d;
    b.in = c->y2;
    b.wt = c->wf[2];
    b.bias = c->p + c->off[5];
    b.out_f32 = out ? out : c->o;
    b.oscale = oscale;
    b.cout_valid = 1;
    if (e == cudaSuccess) {  // the one-channel last layer: tap-split tcgen05 (impl 0), CUDA cores (impl 2)
        if (c->conv_impl == 0)
            e = launch_conv_out1_tc(b, c->derr, c->stream);
        else
            e = c->conv_impl == 2 ? launch_conv_out1(b, c->stream) : conv<8, EPI_LINEAR_F32>(c, b);
    }
    return e == cudaSuccess ? GBST_OK : record_error(GBST_ECUDA, cudaGetErrorString(e));
}

// Backward pass from c->dout (the cotangent of o, channel 0) through the three layers:
// adds every parameter's gradient into c->g; with input_grad, also the cotangent of the
// network input into c->dx.  Needs the activations of forward(.., keep = true).
cudaError_t backprop(gbst_closure c, Dims d, bool input_grad)
{
    cudaStream_t s = c->stream;
    // layer 3: dW3 from y2 and dOut; dZ2 = conv(dOut, W3 flipped^T) * GELU'(z2)
    WgradArgs w{};
    w.d = d;
    w.x = c->y2;
    w.dz = c->dout;
    w.grad_w = c->g + c->off[4];
    w.grad_b = c->g + c->off[5];
    w.cin = c->hidden;
    w.cout = 1;
    cudaError_t e = c->layer_grad[2] ? launch_wgrad(w, s) : cudaSuccess;
    ConvArgs a{};
    a.d = d;
    a.in = c->dout;
    a.wt = c->wb[2];
    a.aux = c->z2;
    a.out = c->dz2;
    a.cout_valid = CH;
    if (e == cudaSuccess)
        e = conv<16, EPI_DGELU>(c, a);
    // layer 2
    w.x = c->y1;
    w.dz = c->dz2;
    w.grad_w = c->g + c->off[2];
    w.grad_b = c->g + c->off[3];
    w.cin = c->hidden;
    w.cout = c->hidden;
    if (e == cudaSuccess && c->layer_grad[1])
        e = launch_wgrad(w, s);
    a.in = c->dz2;
    a.wt = c->wb[1];
    a.aux = c->z1;
    a.out = c->dz1;
    if (e == cudaSuccess)
        e = conv<16, EPI_DGELU>(c, a);
    // layer 1
    w.x = c->x;
    w.dz = c->dz1;
    w.grad_w = c->g + c->off[0];
    w.grad_b = c->g + c->off[1];
    w.cin = c->cin;
    w.cout = c->hidden;
    if (e == cudaSuccess && c->layer_grad[0])
        e = launch_wgrad(w, s);
    if (input_grad && e == cudaSuccess) {
        a.in = c->dz1;
        a.wt = c->wb[0];
        a.aux = nullptr;
        a.bias = nullptr;
        a.out = c->dx;
        e = conv<16, EPI_LINEAR_BF16>(c, a);
    }
    if (e == cudaSuccess)
        e = cudaGetLastError();
    return e;
}

}  // namespace

extern "C" {

gbst_status closure_create(int cin, int hidden, int64_t max_points, double in_scale, void *stream,
                           const gbst_allocator *allocator, gbst_closure *out)
{
    if (!out)
        return record_error(GBST_EINVAL, "closure_create: null out");
    *out = nullptr;
    if ((cin != 4 && cin != 8) || hidden != 16)
        return record_error(GBST_ENOTSUP,
                            "closure_create: the network has 4 (fields) or 8 (fields and FP32 stencil features) "
                            "input channels and 16 hidden channels");
    if (max_points < 1 || !(in_scale > 0.0))
        return record_error(GBST_EINVAL, "closure_create: max_points and in_scale must be positive");
    gbst_closure c = new (std::nothrow) gbst_closure_s;
    if (!c)
        return record_error(GBST_ENOMEM, "closure_create: handle");
    c->cin = cin;
    c->hidden = hidden;
    c->max_pts = max_points;
    c->scale = in_scale;
    c->out_scale = in_scale;
    c->stream = static_cast<cudaStream_t>(stream);
    if (allocator) {
        c->alloc = *allocator;
        c->custom = true;
    }
    const int64_t counts[6] = {int64_t(hidden) * cin * 27, hidden, int64_t(hidden) * hidden * 27, hidden,
                               int64_t(hidden) * 27, 1};
    int64_t o = 0;
    for (int i = 0; i < 6; ++i) {
        c->off[i] = o;
        c->cnt[i] = counts[i];
        o += counts[i];
    }
    c->nparams = o;
    const size_t pb = static_cast<size_t>(o) * sizeof(float);
    const size_t ab = static_cast<size_t>(max_points) * CH * sizeof(__nv_bfloat16);
    c->p = static_cast<float *>(cl_alloc(c, pb));
    c->g = static_cast<float *>(cl_alloc(c, pb));
    c->m1 = static_cast<float *>(cl_alloc(c, pb));
    c->m2 = static_cast<float *>(cl_alloc(c, pb));
    for (int l = 0; l < 3; ++l) {
        c->wf[l] = static_cast<__nv_bfloat16 *>(cl_alloc(c, 27 * CH * CH * sizeof(__nv_bfloat16)));
        c->wb[l] = static_cast<__nv_bfloat16 *>(cl_alloc(c, 27 * CH * CH * sizeof(__nv_bfloat16)));
    }
    __nv_bfloat16 **acts[8] = {&c->x, &c->z1, &c->y1, &c->z2, &c->y2, &c->dout, &c->dz2, &c->dz1};
    bool ok = c->p && c->g && c->m1 && c->m2;
    for (int l = 0; l < 3; ++l)
        ok = ok && c->wf[l] && c->wb[l];
    for (auto pp : acts) {
        *pp = static_cast<__nv_bfloat16 *>(cl_alloc(c, ab));
        ok = ok && *pp;
    }
    if (cin == 8) {
        c->feat = true;
        const size_t fbytes = static_cast<size_t>(max_points) * sizeof(float);
        float **fbufs[9] = {&c->fb.cn2, &c->fb.g[0], &c->fb.g[1], &c->fb.g[2], &c->fb.lu,
                            &c->fb.t5,  &c->fb.t6,   &c->fb.e7,   &c->fb.tmp};
        for (auto pp : fbufs) {
            *pp = static_cast<float *>(cl_alloc(c, fbytes));
            ok = ok && *pp;
        }
        c->dx = static_cast<__nv_bfloat16 *>(cl_alloc(c, ab));
        ok = ok && c->dx;
        double w[9];
        stencil_fd_weights(4, w);
        for (int m = 0; m <= 2; ++m)
            c->feat_w[m] = w[m];
    }
    c->o = static_cast<float *>(cl_alloc(c, static_cast<size_t>(max_points) * sizeof(float)));
    c->dloss = static_cast<double *>(cl_alloc(c, 256));
    c->derr = static_cast<int *>(cl_alloc(c, 256));
    ok = ok && c->o && c->dloss && c->derr;
    if (ok)
        ok = cudaMemsetAsync(c->p, 0, pb, c->stream) == cudaSuccess && cudaMemsetAsync(c->g, 0, pb, c->stream) ==
             cudaSuccess && cudaMemsetAsync(c->m1, 0, pb, c->stream) == cudaSuccess &&
             cudaMemsetAsync(c->m2, 0, pb, c->stream) == cudaSuccess &&
             cudaMemsetAsync(c->derr, 0, 256, c->stream) == cudaSuccess;
    if (!ok) {
        closure_destroy(c);
        return record_error(GBST_ENOMEM, "closure_create: device memory");
    }
    *out = c;
    return GBST_OK;
}

gbst_status closure_destroy(gbst_closure c)
{
    if (!c)
        return GBST_OK;
    cudaStreamSynchronize(c->stream);
    for (auto &pb : c->owned) {
        if (c->custom)
            c->alloc.release(pb.first, pb.second, c->stream, c->alloc.ctx);
        else
            cudaFree(pb.first);
    }
    delete c;
    return GBST_OK;
}

gbst_status closure_param_count(gbst_closure c, int64_t *n)
{
    if (!c || !n)
        return record_error(GBST_EINVAL, "closure_param_count: null argument");
    *n = c->nparams;
    return GBST_OK;
}

gbst_status closure_set_params(gbst_closure c, const float *host, int64_t n)
{
    if (!c || !host || n != c->nparams)
        return record_error(GBST_EINVAL, "closure_set_params: null argument or wrong count");
    if (cudaMemcpyAsync(c->p, host, n * sizeof(float), cudaMemcpyHostToDevice, c->stream) != cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess)
        return record_error(GBST_ECUDA, "closure_set_params: copy failed");
    c->weights_dirty = true;
    return GBST_OK;
}

static gbst_status copy_out(gbst_closure c, const float *src, float *host, int64_t n)
{
    if (!c || !host || n != c->nparams)
        return record_error(GBST_EINVAL, "closure: null argument or wrong count");
    if (cudaMemcpyAsync(host, src, n * sizeof(float), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess)
        return record_error(GBST_ECUDA, "closure: copy failed");
    return check_device_error(c);
}

gbst_status closure_get_params(gbst_closure c, float *host, int64_t n) { return copy_out(c, c->p, host, n); }
gbst_status closure_get_grads(gbst_closure c, float *host, int64_t n) { return copy_out(c, c->g, host, n); }

gbst_status closure_forward(gbst_closure c, const float *u_plus, const float *u_n, const float *c_norm, int64_t nx,
                            int64_t ny, int64_t nz, float *correction)
{
    if (!c || !u_plus || !u_n || !c_norm || !correction)
        return record_error(GBST_EINVAL, "closure_forward: null argument");
    Dims d;
    gbst_status st = check_dims(c, nx, ny, nz, &d);
    if (st != GBST_OK)
        return st;
    // the last layer writes o / t into correction
    return forward(c, u_plus, u_n, c_norm, d, false, correction, static_cast<float>(1.0 / c->out_scale));
}

gbst_status closure_loss_grad(gbst_closure c, const float *u_plus, const float *u_n, const float *c_norm,
                              const float *u_ref, int64_t nx, int64_t ny, int64_t nz, double *loss)
{
    if (!c || !u_plus || !u_n || !c_norm || !u_ref || !loss)
        return record_error(GBST_EINVAL, "closure_loss_grad: null argument");
    Dims d;
    gbst_status st = check_dims(c, nx, ny, nz, &d);
    if (st != GBST_OK)
        return st;
    st = forward(c, u_plus, u_n, c_norm, d, true);
    if (st != GBST_OK)
        return st;
    const int64_t n = nx * ny * nz;
    cudaStream_t s = c->stream;
    cudaError_t e = cudaMemsetAsync(c->dloss, 0, sizeof(double), s);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(c->g, 0, c->nparams * sizeof(float), s);
    k_loss<<<blocks_for(n), 256, 0, s>>>(c->o, u_plus, u_ref, static_cast<float>(c->out_scale),
                                         static_cast<float>(c->loss_weight), n, c->dloss, c->dout);
    if (e == cudaSuccess)
        e = backprop(c, d, false);
    double l = 0.0;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&l, c->dloss, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(s);
    if (e != cudaSuccess)
        return record_error(GBST_ECUDA, cudaGetErrorString(e));
    st = check_device_error(c);
    if (st != GBST_OK)
        return st;
    *loss = c->loss_weight * l / static_cast<double>(n);
    return GBST_OK;
}

gbst_status closure_set_trainable(gbst_closure c, const unsigned char *mask, int64_t n)
{
    if (!c)
        return record_error(GBST_EINVAL, "closure_set_trainable: null closure");
    if (!mask) {
        c->trainable = nullptr;  // (the buffer, if any, stays owned by the closure)
        for (bool &b : c->layer_grad)
            b = true;
        return GBST_OK;
    }
    if (n != c->nparams)
        return record_error(GBST_EINVAL, "closure_set_trainable: n must be the parameter count");
    // a layer whose weights and biases are all frozen needs no weight gradient (its data
    // gradient still flows to the layers below and to the input)
    for (int l = 0; l < 3; ++l) {
        bool any = false;
        for (int64_t i = c->off[2 * l]; i < c->off[2 * l + 1] + c->cnt[2 * l + 1] && !any; ++i)
            any = mask[i] != 0;
        c->layer_grad[l] = any;
    }
    if (!c->trainable_buf) {
        c->trainable_buf = static_cast<unsigned char *>(cl_alloc(c, static_cast<size_t>(n)));
        if (!c->trainable_buf)
            return record_error(GBST_ENOMEM, "closure_set_trainable: device memory");
    }
    if (cudaMemcpyAsync(c->trainable_buf, mask, static_cast<size_t>(n), cudaMemcpyHostToDevice, c->stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess)
        return record_error(GBST_ECUDA, "closure_set_trainable: copy failed");
    c->trainable = c->trainable_buf;
    return GBST_OK;
}

gbst_status closure_set_features(gbst_closure c, int space_order, const double *scales, int n)
{
    if (!c || !scales || n != 8)
        return record_error(GBST_EINVAL, "closure_set_features: null closure or scales, or n != 8");
    if (!c->feat)
        return record_error(GBST_ENOTSUP, "closure_set_features: the closure was created with 4 input channels");
    if (space_order != 2 && space_order != 4 && space_order != 8)
        return record_error(GBST_EINVAL, "closure_set_features: space_order must be 2, 4 or 8");
    for (int k = 0; k < 8; ++k)
        if (!std::isfinite(scales[k]))
            return record_error(GBST_EINVAL, "closure_set_features: scales must be finite");
    double w[9];
    gbst_status st = stencil_fd_weights(space_order, w);
    if (st != GBST_OK)
        return st;
    c->feat_r = space_order / 2;
    for (int m = 0; m < 5; ++m)
        c->feat_w[m] = m <= c->feat_r ? w[m] : 0.0;
    for (int k = 0; k < 8; ++k)
        c->feat_s[k] = scales[k];
    return GBST_OK;
}

gbst_status closure_gelu(const float *x, float *y, int64_t n, void *stream)
{
    if (!x || !y || n < 0)
        return record_error(GBST_EINVAL, "closure_gelu: null array or n < 0");
    if (n == 0)
        return GBST_OK;
    k_gelu<<<blocks_for(n), 256, 0, static_cast<cudaStream_t>(stream)>>>(x, y, n);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? GBST_OK : record_error(GBST_ECUDA, cudaGetErrorString(e));
}

gbst_status closure_feature_values(gbst_closure c, const float *u_plus, const float *u_n, const float *c_norm,
                                   int64_t nx, int64_t ny, int64_t nz, float *out)
{
    if (!c || !u_plus || !u_n || !c_norm || !out)
        return record_error(GBST_EINVAL, "closure_feature_values: null argument");
    if (!c->feat)
        return record_error(GBST_ENOTSUP, "closure_feature_values: the closure was created with 4 input channels");
    Dims d;
    gbst_status st = check_dims(c, nx, ny, nz, &d);
    if (st != GBST_OK)
        return st;
    st = closure_features_forward(u_plus, u_n, c_norm, nx, ny, nz, c->feat_r, c->feat_w, c->feat_s, c->fb, c->x,
                                  true, 16, c->stream);
    if (st != GBST_OK)
        return st;
    return closure_features_values(u_plus, u_n, nx, ny, nz, c->fb, out, c->stream);
}

gbst_status closure_backward(gbst_closure c, const float *u_plus, const float *u_n, const float *c_norm,
                             int64_t nx, int64_t ny, int64_t nz, const float *grad_out, float *grad_up,
                             float *grad_un, int accumulate)
{
    const float *grad_corr = grad_out;
    if (!c || !u_plus || !u_n || !c_norm || !grad_corr || !grad_up || !grad_un || grad_up == grad_out)
        return record_error(GBST_EINVAL, "closure_backward: null argument");
    if (!c->feat)
        return record_error(GBST_ENOTSUP, "closure_backward: the closure was created with 4 input channels");
    Dims d;
    gbst_status st = check_dims(c, nx, ny, nz, &d);
    if (st != GBST_OK)
        return st;
    st = forward(c, u_plus, u_n, c_norm, d, true);
    if (st != GBST_OK)
        return st;
    const int64_t n = nx * ny * nz;
    cudaError_t e = cudaSuccess;
    if (!accumulate)
        e = cudaMemsetAsync(c->g, 0, c->nparams * sizeof(float), c->stream);
    k_seed<<<blocks_for(n), 256, 0, c->stream>>>(grad_corr, static_cast<float>(1.0 / c->out_scale), n, c->dout);
    if (e == cudaSuccess)
        e = backprop(c, d, true);
    if (e != cudaSuccess)
        return record_error(GBST_ECUDA, cudaGetErrorString(e));
    st = closure_features_adjoint(c->dx, nx, ny, nz, c->feat_r, c->feat_w, c->feat_s, c->fb, grad_up, grad_un,
                                  c->stream);
    if (st != GBST_OK)
        return st;
    // u^{n+1} = u+ + correction: the identity path of u+
    k_scale_add<<<blocks_for(n), 256, 0, c->stream>>>(grad_up, grad_out, 1.0f, n);
    e = cudaGetLastError();
    return e == cudaSuccess ? GBST_OK : record_error(GBST_ECUDA, cudaGetErrorString(e));
}

gbst_status closure_set_out_scale(gbst_closure c, double out_scale)
{
    if (!c || !(out_scale > 0.0))
        return record_error(GBST_EINVAL, "closure_set_out_scale: null closure or scale <= 0");
    c->out_scale = out_scale;
    return GBST_OK;
}

gbst_status closure_set_loss_weight(gbst_closure c, double w)
{
    if (!c || !(w > 0.0))
        return record_error(GBST_EINVAL, "closure_set_loss_weight: null closure or weight <= 0");
    c->loss_weight = w;
    return GBST_OK;
}

gbst_status closure_set_conv_impl(gbst_closure c, int impl)
{
    if (!c || impl < 0 || impl > 3)
        return record_error(GBST_EINVAL, "closure_set_conv_impl: null closure or impl not 0, 1, 2 or 3");
    c->conv_impl = impl;
    return GBST_OK;
}

gbst_status closure_freeze_biases(gbst_closure c, int freeze)
{
    if (!c)
        return record_error(GBST_EINVAL, "closure_freeze_biases: null closure");
    c->freeze_biases = freeze != 0;
    return GBST_OK;
}

gbst_status closure_adam_step(gbst_closure c, double lr)
{
    if (!c || !(lr > 0.0))
        return record_error(GBST_EINVAL, "closure_adam_step: null closure or lr <= 0");
    c->t += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float bc1 = static_cast<float>(1.0 - std::pow(0.9, static_cast<double>(c->t)));
    const float bc2 = static_cast<float>(1.0 - std::pow(0.999, static_cast<double>(c->t)));
    BiasRanges fr{};
    for (int l = 0; l < 3; ++l) {
        fr.lo[l] = c->freeze_biases ? static_cast<int>(c->off[2 * l + 1]) : 0;
        fr.hi[l] = c->freeze_biases ? static_cast<int>(c->off[2 * l + 1] + c->cnt[2 * l + 1]) : 0;
    }
    k_adam<<<blocks_for(c->nparams), 256, 0, c->stream>>>(c->p, c->g, c->m1, c->m2, static_cast<int>(c->nparams),
                                                          static_cast<float>(lr), b1, b2, static_cast<float>(1.0 - 0.9),
                                                          static_cast<float>(1.0 - 0.999), 1e-8f, bc1, bc2, fr,
                                                          c->trainable);
    c->weights_dirty = true;
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? GBST_OK : record_error(GBST_ECUDA, cudaGetErrorString(e));
}

}  // extern "C"
