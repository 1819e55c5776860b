// Dense-array stencil kernels that train and feed the learned closure.
//
// The closure works on dense [nz][ny][nx] FP32 arrays (x fastest) of one coarse
// grid, zero outside the interior.  Training it through whole coarse-grid
// rollouts needs the transpose of the leapfrog step of Section 6.1's scheme
// (backpropagation through the time steps), and its input features are
// stencils of the field computed in FP32 before they are rounded to the
// network's BF16 inputs.  These kernels are simple one-thread-per-point
// stencils: each output point reads its star neighbours (L2-resident at the
// closure's grid sizes), so they cost a few tens of microseconds at 256^3,
// small next to the network.
#include <cmath>
#include <cstdio>

#include "gbst_internal.h"

namespace gbst {
namespace {

struct DenseDims {
    int nx, ny, nz;
};

struct FeatScales {
    float s[8];
};

constexpr int kThr = 256;

inline int blocks_for_dense(int64_t n) { return static_cast<int>(std::min<int64_t>(65535 * 8, (n + kThr - 1) / kThr)); }

// Stencil kernels: threads along x, blocks over (x segments, y, z), so that no
// point pays an integer division for its coordinates.
constexpr int kDX = 128;
inline dim3 dense_grid(const DenseDims &d)
{
    return dim3(static_cast<unsigned>((d.nx + kDX - 1) / kDX), static_cast<unsigned>(std::min(d.ny, 65535)),
                static_cast<unsigned>(std::min(d.nz, 65535)));
}
// Every interior point (x, y, z) of d once, with its linear index p, over dense_grid(d).
#define GBST_DENSE_POINTS(d)                                                                                   \
    for (int z = blockIdx.z; z < (d).nz; z += gridDim.z)                                                       \
        for (int y = blockIdx.y; y < (d).ny; y += gridDim.y)                                                   \
            for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < (d).nx; x += gridDim.x * blockDim.x)       \
                if (const int64_t p = (static_cast<int64_t>(z) * (d).ny + y) * (d).nx + x; true)

// out[p] (=|+=) alpha * post[p] * sum_axes sum_{m=-R..R} w_|m| (pre * in)[p + m e_axis]
// with zero outside the interior; pre / post may be null (factor 1).
template <int R>
__global__ void __launch_bounds__(kThr) k_star(DenseDims d, const float *__restrict__ in,
                                               const float *__restrict__ pre, const float *__restrict__ post,
                                               float4 w03, float w4, float alpha, int accumulate,
                                               float *__restrict__ out)
{
    const float w[5] = {w03.x, w03.y, w03.z, w03.w, w4};
    const int64_t sy = d.nx, sz = static_cast<int64_t>(d.nx) * d.ny;
    GBST_DENSE_POINTS(d) {
        auto val = [&](int64_t q) { return pre ? pre[q] * in[q] : in[q]; };
        float s = 3.0f * w[0] * val(p);
#pragma unroll
        for (int m = 1; m <= R; ++m) {
            float a = 0.0f;
            if (x - m >= 0) a += val(p - m);
            if (x + m < d.nx) a += val(p + m);
            if (y - m >= 0) a += val(p - m * sy);
            if (y + m < d.ny) a += val(p + m * sy);
            if (z - m >= 0) a += val(p - m * sz);
            if (z + m < d.nz) a += val(p + m * sz);
            s = fmaf(w[m], a, s);
        }
        float v = alpha * s;
        if (post)
            v *= post[p];
        out[p] = accumulate ? out[p] + v : v;
    }
}

// Transpose of one source-free leapfrog step:
//   lam_cur += 2 lam_next + L(kappa lam_next);  lam_prev = -lam_next (when given).
template <int R>
__global__ void __launch_bounds__(kThr) k_wave_adjoint(DenseDims d, const float *__restrict__ kappa,
                                                       const float *__restrict__ lam_next, float4 w03, float w4,
                                                       float *__restrict__ lam_cur, float *__restrict__ lam_prev)
{
    const float w[5] = {w03.x, w03.y, w03.z, w03.w, w4};
    const int64_t sy = d.nx, sz = static_cast<int64_t>(d.nx) * d.ny;
    GBST_DENSE_POINTS(d) {
        auto val = [&](int64_t q) { return kappa[q] * lam_next[q]; };
        float s = 3.0f * w[0] * val(p);
#pragma unroll
        for (int m = 1; m <= R; ++m) {
            float a = 0.0f;
            if (x - m >= 0) a += val(p - m);
            if (x + m < d.nx) a += val(p + m);
            if (y - m >= 0) a += val(p - m * sy);
            if (y + m < d.ny) a += val(p + m * sy);
            if (z - m >= 0) a += val(p - m * sz);
            if (z + m < d.nz) a += val(p + m * sz);
            s = fmaf(w[m], a, s);
        }
        const float ln = lam_next[p];
        lam_cur[p] = lam_cur[p] + (2.0f * ln + s);
        if (lam_prev)
            lam_prev[p] = -ln;
    }
}

// Value of a dense array at p + m e_axis, zero outside the interior.
__device__ __forceinline__ float at_off(const float *__restrict__ u, DenseDims d, int64_t p, int x, int y, int z,
                                        int axis, int m)
{
    if (axis == 0)
        return (x + m >= 0 && x + m < d.nx) ? u[p + m] : 0.0f;
    if (axis == 1)
        return (y + m >= 0 && y + m < d.ny) ? u[p + static_cast<int64_t>(m) * d.nx] : 0.0f;
    return (z + m >= 0 && z + m < d.nz) ? u[p + static_cast<int64_t>(m) * d.nx * d.ny] : 0.0f;
}

// cn2 = c_n^2 and its central differences g_a = (cn2[p + e_a] - cn2[p - e_a]) / 2 (zero outside).
__global__ void __launch_bounds__(kThr) k_cn2_grads(DenseDims d, const float *__restrict__ cn, float *__restrict__ cn2,
                                                    float *__restrict__ g0, float *__restrict__ g1,
                                                    float *__restrict__ g2)
{
    GBST_DENSE_POINTS(d) {
        const float c = cn[p];
        cn2[p] = c * c;
        float *g[3] = {g0, g1, g2};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float cp = at_off(cn, d, p, x, y, z, a, 1), cm = at_off(cn, d, p, x, y, z, a, -1);
            g[a][p] = 0.5f * (cp * cp - cm * cm);
        }
    }
}

// Network input x (channels-last BF16, 16 channels) from the FP32 features:
//   f0 = u+, f1 = u^n, f2 = cn2 u+, f3 = cn2 u^n, f4 = t6 (= cn2 sum delta^6 u^n),
//   f5 = t5 (= cn2 L(cn2 L u^n)), f6 = sum_a g_a D_a u^n, f7 = (sum_a |g_a|) Lu;  x_k = s_k f_k.
__global__ void __launch_bounds__(kThr) k_pack_features(DenseDims d, const float *__restrict__ up,
                                                        const float *__restrict__ un, const float *__restrict__ cn2,
                                                        const float *__restrict__ t6, const float *__restrict__ t5,
                                                        const float *__restrict__ lu, const float *__restrict__ g0,
                                                        const float *__restrict__ g1, const float *__restrict__ g2,
                                                        FeatScales sc, __nv_bfloat16 *__restrict__ xout)
{
    GBST_DENSE_POINTS(d) {
        const float c2 = cn2[p], a = up[p], b = un[p];
        const float ga[3] = {g0[p], g1[p], g2[p]};
        float f6 = 0.0f, gabs = 0.0f;
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) {
            const float du = 0.5f * (at_off(un, d, p, x, y, z, ax, 1) - at_off(un, d, p, x, y, z, ax, -1));
            f6 = fmaf(ga[ax], du, f6);
            gabs += fabsf(ga[ax]);
        }
        const float f[8] = {a, b, c2 * a, c2 * b, t6[p], t5[p], f6, gabs * lu[p]};
        uint32_t w4[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const __nv_bfloat162 b2 = __floats2bfloat162_rn(sc.s[2 * k] * f[2 * k], sc.s[2 * k + 1] * f[2 * k + 1]);
            w4[k] = *reinterpret_cast<const uint32_t *>(&b2);
        }
        // channels 0-7, then 8-15 (zero): two 16-byte stores
        uint4 *o = reinterpret_cast<uint4 *>(xout + p * 16);
        o[0] = make_uint4(w4[0], w4[1], w4[2], w4[3]);
        o[1] = make_uint4(0u, 0u, 0u, 0u);
    }
}

// z-marching forms of the forward features (inference): a block owns a 32 x 8
// (x, y) tile and a chunk of kFZC planes, each thread one column; the z
// neighbours of the star stencils come from register queues (one new load per
// plane and field), the x and y neighbours from L1 (lu) or from shared-memory
// plane tiles (the features).  Same arithmetic, in the same order, as k_star /
// k_cn2_grads / k_pack_features.
constexpr int kFX = 32, kFY = 8, kFZC = 32;
inline dim3 zmarch_grid(const DenseDims &d)
{
    return dim3(static_cast<unsigned>((d.nx + kFX - 1) / kFX), static_cast<unsigned>((d.ny + kFY - 1) / kFY),
                static_cast<unsigned>((d.nz + kFZC - 1) / kFZC));
}

// Plane tiles in shared memory for the z-marching feature kernel: element e of a W x H
// tile (halo h around the block's kFX x kFY points) is staged by thread e mod
// (kFX kFY), at an offset within a plane fixed for the whole z-march (-1: outside
// the grid, staged as 0; -2: no element).  The next plane's values are loaded into
// registers before the current plane is computed and stored to the other buffer
// after it, one barrier per plane.
template <int W, int H>
struct PlaneTile {
    static constexpr int NT = kFX * kFY, NE = W * H, K = (NE + NT - 1) / NT;
    int off[K];
    __device__ void init(const DenseDims &d, int bx, int by, int h, int tid)
    {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int e = tid + k * NT;
            const int gx = bx - h + e % W, gy = by - h + e / W;
            off[k] = e >= NE ? -2 : (gx >= 0 && gx < d.nx && gy >= 0 && gy < d.ny) ? gy * d.nx + gx : -1;
        }
    }
};

// lu = L u^n (star of radius R, weights w), as k_star with no pre / post factor.
template <int R>
__global__ void __launch_bounds__(kFX *kFY) k_lap_z(DenseDims d, const float *__restrict__ un, float4 w03, float w4,
                                                    float *__restrict__ lu)
{
    const float w[5] = {w03.x, w03.y, w03.z, w03.w, w4};
    const int x = blockIdx.x * kFX + threadIdx.x, y = blockIdx.y * kFY + threadIdx.y;
    if (x >= d.nx || y >= d.ny)
        return;
    const int z0 = blockIdx.z * kFZC, z1 = min(d.nz, z0 + kFZC);
    const int64_t sy = d.nx, sz = static_cast<int64_t>(d.nx) * d.ny, pxy = static_cast<int64_t>(y) * d.nx + x;
    float q[2 * R + 1];  // u^n at z - R .. z + R (zero outside)
#pragma unroll
    for (int k = 0; k < 2 * R + 1; ++k) {
        const int zz = z0 - R + k;
        q[k] = (zz >= 0 && zz < d.nz) ? un[zz * sz + pxy] : 0.0f;
    }
    for (int z = z0; z < z1; ++z) {
        const int64_t p = z * sz + pxy;
        float s = 3.0f * w[0] * q[R];
#pragma unroll
        for (int m = 1; m <= R; ++m) {
            float a = 0.0f;
            if (x - m >= 0) a += un[p - m];
            if (x + m < d.nx) a += un[p + m];
            if (y - m >= 0) a += un[p - m * sy];
            if (y + m < d.ny) a += un[p + m * sy];
            if (z - m >= 0) a += q[R - m];
            if (z + m < d.nz) a += q[R + m];
            s = fmaf(w[m], a, s);
        }
        lu[p] = s;
#pragma unroll
        for (int k = 0; k < 2 * R; ++k)
            q[k] = q[k + 1];
        q[2 * R] = (z + R + 1 < d.nz) ? un[p + (R + 1) * sz] : 0.0f;
    }
}

// lu = L u^n as k_lap_z (the same sums in the same order, so the same bits), four
// consecutive x points per thread (rows a multiple of 4 points, 16-byte aligned arrays):
// a block owns a 128 x 8 (x, y) tile and a chunk of kFZC planes; the own points and
// the y neighbours are 16-byte loads, the x neighbours outside the thread's four points
// 8- or 16-byte loads, the z neighbours a register queue of 2R + 1 planes whose slots
// are compile-time constants (the z-loop unrolled by 2R + 1).  Points outside the grid
// read as 0, which adds nothing to a sum that starts at 0 (k_lap_z skips them).
template <int R>
__global__ void __launch_bounds__(kFX *kFY) k_lap4_z(DenseDims d, const float *__restrict__ un, float4 w03,
                                                     float w4, float *__restrict__ lu)
{
    constexpr int QN = 2 * R + 1;
    const float w[5] = {w03.x, w03.y, w03.z, w03.w, w4};
    const int x0 = (blockIdx.x * kFX + threadIdx.x) * 4, y = blockIdx.y * kFY + threadIdx.y;
    if (x0 >= d.nx || y >= d.ny)
        return;
    const int z0 = blockIdx.z * kFZC, z1 = min(d.nz, z0 + kFZC);
    const int64_t sy = d.nx, sz = static_cast<int64_t>(d.nx) * d.ny, pxy = static_cast<int64_t>(y) * d.nx + x0;
    const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
    auto ld4 = [&](int64_t p) { return *reinterpret_cast<const float4 *>(un + p); };
    float4 q[QN];  // u^n at planes z - R .. z + R of the thread's four points (slot = plane mod QN)
#pragma unroll
    for (int k = 0; k < 2 * R; ++k) {
        const int zz = z0 - R + k;
        q[(k + QN - R) % QN] = (zz >= 0 && zz < d.nz) ? ld4(zz * sz + pxy) : zero4;
    }
    for (int c0 = z0; c0 < z1; c0 += QN) {
#pragma unroll
        for (int k = 0; k < QN; ++k) {
            const int z = c0 + k;
            if (z < z1) {
                // plane z + R into its slot; the slot of plane z is k mod QN (c0 - z0 is a multiple of QN)
                const int zn = z + R;
                q[(k + R) % QN] = zn < d.nz ? ld4(zn * sz + pxy) : zero4;
                const int64_t p = z * sz + pxy;
                const float4 c = q[k % QN];
                const float cv[4] = {c.x, c.y, c.z, c.w};
                // x neighbours: elements x0 - R .. x0 - 1 and x0 + 4 .. x0 + 3 + R
                float xl[4] = {0.f, 0.f, 0.f, 0.f}, xr[4] = {0.f, 0.f, 0.f, 0.f};
                if (x0 > 0) {
                    if (R <= 2) {
                        const float2 t = *reinterpret_cast<const float2 *>(un + p - 2);
                        xl[2] = t.x;
                        xl[3] = t.y;
                    } else {
                        const float4 t = ld4(p - 4);
                        xl[0] = t.x;
                        xl[1] = t.y;
                        xl[2] = t.z;
                        xl[3] = t.w;
                    }
                }
                if (x0 + 4 < d.nx) {
                    if (R <= 2) {
                        const float2 t = *reinterpret_cast<const float2 *>(un + p + 4);
                        xr[0] = t.x;
                        xr[1] = t.y;
                    } else {
                        const float4 t = ld4(p + 4);
                        xr[0] = t.x;
                        xr[1] = t.y;
                        xr[2] = t.z;
                        xr[3] = t.w;
                    }
                }
                // element e in [-4, 8) of the thread's row
                auto xe = [&](int e) { return e < 0 ? xl[4 + e] : e >= 4 ? xr[e - 4] : cv[e]; };
                float4 ym[R], yp[R];
#pragma unroll
                for (int m = 1; m <= R; ++m) {
                    ym[m - 1] = y - m >= 0 ? ld4(p - m * sy) : zero4;
                    yp[m - 1] = y + m < d.ny ? ld4(p + m * sy) : zero4;
                }
                float o[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    float s = 3.0f * w[0] * cv[i];
#pragma unroll
                    for (int m = 1; m <= R; ++m) {
                        const float yl[4] = {ym[m - 1].x, ym[m - 1].y, ym[m - 1].z, ym[m - 1].w};
                        const float yh[4] = {yp[m - 1].x, yp[m - 1].y, yp[m - 1].z, yp[m - 1].w};
                        const float4 zl = q[(k - m + 2 * QN) % QN], zh = q[(k + m) % QN];
                        const float zlv[4] = {zl.x, zl.y, zl.z, zl.w}, zhv[4] = {zh.x, zh.y, zh.z, zh.w};
                        float a = 0.0f;
                        a += xe(i - m);
                        a += xe(i + m);
                        a += yl[i];
                        a += yh[i];
                        a += zlv[i];
                        a += zhv[i];
                        s = fmaf(w[m], a, s);
                    }
                    o[i] = s;
                }
                *reinterpret_cast<float4 *>(lu + p) = make_float4(o[0], o[1], o[2], o[3]);
            }
        }
    }
}

// The packed network input from u+, u^n, c_n and lu = L u^n: cn2 and g_a as
// k_cn2_grads, t6 and t5 as the k_star calls of closure_features_forward, the
// channels as k_pack_features.  R: the radius of L; w6: the sixth-difference star;
// XCH: channels per point of x (16: the last 8 zero; 8: packed, 16 bytes per point).
// The x and y neighbours come from plane tiles of u^n (halo 3: sixth differences,
// D_a) and of c_n and c_n^2 lu (halo R: t5, g_a), zero outside the grid (an absent
// neighbour adds 0 where the dense kernels skip it: the same sums).
template <int R, int XCH>
__global__ void __launch_bounds__(kFX *kFY) k_features_z(DenseDims d, const float *__restrict__ up,
                                                         const float *__restrict__ un, const float *__restrict__ cn,
                                                         const float *__restrict__ lu, float4 w03, float w4,
                                                         float4 w6, FeatScales sc, __nv_bfloat16 *__restrict__ xout)
{
    constexpr int QC = R;  // queue radius of c_n and lu (R >= 1 also covers the gradients)
    constexpr int HU = 3, UW = kFX + 2 * HU, UH = kFY + 2 * HU;  // u^n tile
    constexpr int HC = R, CW = kFX + 2 * HC, CH = kFY + 2 * HC;  // c_n and c_n^2 lu tiles
    using TU = PlaneTile<UW, UH>;
    using TC = PlaneTile<CW, CH>;
    __shared__ float su[2][TU::NE], scn[2][TC::NE], scl[2][TC::NE];
    const float w[5] = {w03.x, w03.y, w03.z, w03.w, w4};
    const float v6[4] = {w6.x, w6.y, w6.z, w6.w};
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * kFX + tx;
    const int bx = blockIdx.x * kFX, by = blockIdx.y * kFY;
    const int x = bx + tx, y = by + ty;
    const bool own = x < d.nx && y < d.ny;  // every thread stages; these compute
    const int z0 = blockIdx.z * kFZC, z1 = min(d.nz, z0 + kFZC);
    const int64_t sz = static_cast<int64_t>(d.nx) * d.ny, pxy = static_cast<int64_t>(y) * d.nx + x;
    TU tu;
    TC tc;
    tu.init(d, bx, by, HU, tid);
    tc.init(d, bx, by, HC, tid);
    float ru[TU::K], rc[TC::K], rl[TC::K];
    auto fetch = [&](int z) {
        const int64_t pz = z * sz;
#pragma unroll
        for (int k = 0; k < TU::K; ++k)
            ru[k] = tu.off[k] >= 0 ? un[pz + tu.off[k]] : 0.0f;
#pragma unroll
        for (int k = 0; k < TC::K; ++k) {
            const bool in = tc.off[k] >= 0;
            rc[k] = in ? cn[pz + tc.off[k]] : 0.0f;
            rl[k] = in ? lu[pz + tc.off[k]] : 0.0f;
        }
    };
    auto store = [&](int b) {
#pragma unroll
        for (int k = 0; k < TU::K; ++k)
            if (tu.off[k] != -2)
                su[b][tid + k * TU::NT] = ru[k];
#pragma unroll
        for (int k = 0; k < TC::K; ++k)
            if (tc.off[k] != -2) {
                scn[b][tid + k * TC::NT] = rc[k];
                scl[b][tid + k * TC::NT] = (rc[k] * rc[k]) * rl[k];
            }
    };
    float qu[7], qc[2 * QC + 1], ql[2 * QC + 1];  // u^n at z - 3 .. z + 3; c_n, lu at z - QC .. z + QC
#pragma unroll
    for (int k = 0; k < 7; ++k) {
        const int zz = z0 - 3 + k;
        qu[k] = (own && zz >= 0 && zz < d.nz) ? un[zz * sz + pxy] : 0.0f;
    }
#pragma unroll
    for (int k = 0; k < 2 * QC + 1; ++k) {
        const int zz = z0 - QC + k;
        const bool in = own && zz >= 0 && zz < d.nz;
        qc[k] = in ? cn[zz * sz + pxy] : 0.0f;
        ql[k] = in ? lu[zz * sz + pxy] : 0.0f;
    }
    fetch(z0);
    store(0);
    __syncthreads();
    const int u0 = (ty + HU) * UW + tx + HU, c0 = (ty + HC) * CW + tx + HC;
    for (int z = z0; z < z1; ++z) {
        const int b = (z - z0) & 1;
        if (z + 1 < z1)
            fetch(z + 1);
        const int64_t p = z * sz + pxy;
        if (own) {
            const float *tu_ = su[b] + u0, *tcn = scn[b] + c0, *tcl = scl[b] + c0;
            const float c = qc[QC], c2 = c * c, a = up[p], bq = qu[3];
            // g_a = (cn2[p + e_a] - cn2[p - e_a]) / 2 and D_a u^n, zero outside
            float ga[3], du[3];
            {
                const float cxp = tcn[1], cxm = tcn[-1], cyp = tcn[CW], cym = tcn[-CW];
                ga[0] = 0.5f * (cxp * cxp - cxm * cxm);
                ga[1] = 0.5f * (cyp * cyp - cym * cym);
                ga[2] = 0.5f * (qc[QC + 1] * qc[QC + 1] - qc[QC - 1] * qc[QC - 1]);
                du[0] = 0.5f * (tu_[1] - tu_[-1]);
                du[1] = 0.5f * (tu_[UW] - tu_[-UW]);
                du[2] = 0.5f * (qu[4] - qu[2]);
            }
            float f6 = 0.0f, gabs = 0.0f;
#pragma unroll
            for (int ax = 0; ax < 3; ++ax) {
                f6 = fmaf(ga[ax], du[ax], f6);
                gabs += fabsf(ga[ax]);
            }
            // t6 = cn2 * sum_axes delta^6 u^n
            float s6 = 3.0f * v6[0] * bq;
#pragma unroll
            for (int m = 1; m <= 3; ++m) {
                float t = 0.0f;
                t += tu_[-m];
                t += tu_[m];
                t += tu_[-m * UW];
                t += tu_[m * UW];
                if (z - m >= 0) t += qu[3 - m];
                if (z + m < d.nz) t += qu[3 + m];
                s6 = fmaf(v6[m], t, s6);
            }
            // t5 = cn2 * L(cn2 lu)
            float s5 = 3.0f * w[0] * (c2 * ql[QC]);
#pragma unroll
            for (int m = 1; m <= R; ++m) {
                float t = 0.0f;
                t += tcl[-m];
                t += tcl[m];
                t += tcl[-m * CW];
                t += tcl[m * CW];
                if (z - m >= 0) t += (qc[QC - m] * qc[QC - m]) * ql[QC - m];
                if (z + m < d.nz) t += (qc[QC + m] * qc[QC + m]) * ql[QC + m];
                s5 = fmaf(w[m], t, s5);
            }
            const float f[8] = {a, bq, c2 * a, c2 * bq, s6 * c2, s5 * c2, f6, gabs * ql[QC]};
            uint32_t w4p[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const __nv_bfloat162 b2 =
                    __floats2bfloat162_rn(sc.s[2 * k] * f[2 * k], sc.s[2 * k + 1] * f[2 * k + 1]);
                w4p[k] = *reinterpret_cast<const uint32_t *>(&b2);
            }
            uint4 *o = reinterpret_cast<uint4 *>(xout + p * XCH);
            o[0] = make_uint4(w4p[0], w4p[1], w4p[2], w4p[3]);
            if (XCH == 16)
                o[1] = make_uint4(0u, 0u, 0u, 0u);
        }
#pragma unroll
        for (int k = 0; k < 6; ++k)
            qu[k] = qu[k + 1];
        qu[6] = (own && z + 4 < d.nz) ? un[p + 4 * sz] : 0.0f;
#pragma unroll
        for (int k = 0; k < 2 * QC; ++k) {
            qc[k] = qc[k + 1];
            ql[k] = ql[k + 1];
        }
        const bool in = own && z + QC + 1 < d.nz;
        qc[2 * QC] = in ? cn[p + (QC + 1) * sz] : 0.0f;
        ql[2 * QC] = in ? lu[p + (QC + 1) * sz] : 0.0f;
        if (z + 1 < z1)
            store(b ^ 1);
        __syncthreads();
    }
}

// The same eight features in FP32, unscaled, channel-major (out + k n).
__global__ void __launch_bounds__(kThr) k_feature_values(DenseDims d, const float *__restrict__ up,
                                                         const float *__restrict__ un, const float *__restrict__ cn2,
                                                         const float *__restrict__ t6, const float *__restrict__ t5,
                                                         const float *__restrict__ lu, const float *__restrict__ g0,
                                                         const float *__restrict__ g1, const float *__restrict__ g2,
                                                         float *__restrict__ out)
{
    GBST_DENSE_POINTS(d) {
        const float c2 = cn2[p], a = up[p], b = un[p];
        const float ga[3] = {g0[p], g1[p], g2[p]};
        float f6 = 0.0f, gabs = 0.0f;
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) {
            const float du = 0.5f * (at_off(un, d, p, x, y, z, ax, 1) - at_off(un, d, p, x, y, z, ax, -1));
            f6 = fmaf(ga[ax], du, f6);
            gabs += fabsf(ga[ax]);
        }
        const float f[8] = {a, b, c2 * a, c2 * b, t6[p], t5[p], f6, gabs * lu[p]};
#pragma unroll
        for (int k = 0; k < 8; ++k)
            out[k * (static_cast<int64_t>(d.nx) * d.ny * d.nz) + p] = f[k];
    }
}

// First pass of the features' transpose, from the cotangent dx of the network input
// (channels-last BF16): d_k = s_k dx_k;
//   g_up = d0 + cn2 d2,  g_un = d1 + cn2 d3  (pointwise parts, written),
//   e4 = cn2 d4, e5 = cn2 d5, e6 = d6, e7 = (sum_a |g_a|) d7  (for the stencil parts).
__global__ void __launch_bounds__(kThr) k_unpack_features_adj(DenseDims d, const __nv_bfloat16 *__restrict__ dx,
                                                              const float *__restrict__ cn2,
                                                              const float *__restrict__ g0,
                                                              const float *__restrict__ g1,
                                                              const float *__restrict__ g2, FeatScales sc,
                                                              float *__restrict__ g_up, float *__restrict__ g_un,
                                                              float *__restrict__ e4, float *__restrict__ e5,
                                                              float *__restrict__ e6, float *__restrict__ e7)
{
    const int64_t n = static_cast<int64_t>(d.nx) * d.ny * d.nz;
    for (int64_t p = blockIdx.x * static_cast<int64_t>(kThr) + threadIdx.x; p < n;
         p += static_cast<int64_t>(gridDim.x) * kThr) {
        const __nv_bfloat162 *q = reinterpret_cast<const __nv_bfloat162 *>(dx + p * 16);
        float v[8];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float2 t = __bfloat1622float2(q[k]);
            v[2 * k] = sc.s[2 * k] * t.x;
            v[2 * k + 1] = sc.s[2 * k + 1] * t.y;
        }
        const float c2 = cn2[p];
        g_up[p] = fmaf(c2, v[2], v[0]);
        g_un[p] = fmaf(c2, v[3], v[1]);
        e4[p] = c2 * v[4];
        e5[p] = c2 * v[5];
        e6[p] = v[6];
        e7[p] = (fabsf(g0[p]) + fabsf(g1[p]) + fabsf(g2[p])) * v[7];
    }
}

// out[p] += alpha * sum_a (D_a (g_a * e))[p],  D_a the central difference, zero outside.
__global__ void __launch_bounds__(kThr) k_div_acc(DenseDims d, const float *__restrict__ e,
                                                  const float *__restrict__ g0, const float *__restrict__ g1,
                                                  const float *__restrict__ g2, float alpha, float *__restrict__ out)
{
    const float *g[3] = {g0, g1, g2};
    GBST_DENSE_POINTS(d) {
        float s = 0.0f;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const int64_t st = a == 0 ? 1 : a == 1 ? d.nx : static_cast<int64_t>(d.nx) * d.ny;
            const int c = a == 0 ? x : a == 1 ? y : z, nc = a == 0 ? d.nx : a == 1 ? d.ny : d.nz;
            const float hi = c + 1 < nc ? g[a][p + st] * e[p + st] : 0.0f;
            const float lo = c - 1 >= 0 ? g[a][p - st] * e[p - st] : 0.0f;
            s += 0.5f * (hi - lo);
        }
        out[p] = fmaf(alpha, s, out[p]);
    }
}

// sums[0] += sum (u - ref)^2, sums[1] += sum ref^2  (FP64, one atomic per warp)
__global__ void __launch_bounds__(kThr) k_roll_sums(const float *__restrict__ u, const float *__restrict__ ref,
                                                    int64_t n, double *sums)
{
    double a = 0.0, b = 0.0;
    for (int64_t p = blockIdx.x * static_cast<int64_t>(kThr) + threadIdx.x; p < n;
         p += static_cast<int64_t>(gridDim.x) * kThr) {
        const double r = ref[p], d = static_cast<double>(u[p]) - r;
        a += d * d;
        b += r * r;
    }
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&sums[0], a);
        atomicAdd(&sums[1], b);
    }
}

// u <- scale * 2 (u - ref) / sums[1]  (the gradient of scale * |u - ref|^2 / |ref|^2)
__global__ void __launch_bounds__(kThr) k_roll_grad(float *__restrict__ u, const float *__restrict__ ref, int64_t n,
                                                    const double *sums, double scale)
{
    const double f = sums[1] > 0.0 ? 2.0 * scale / sums[1] : 0.0;
    for (int64_t p = blockIdx.x * static_cast<int64_t>(kThr) + threadIdx.x; p < n;
         p += static_cast<int64_t>(gridDim.x) * kThr)
        u[p] = static_cast<float>(f * (static_cast<double>(u[p]) - ref[p]));
}

__global__ void __launch_bounds__(kThr) k_axpy(float *__restrict__ y, const float *__restrict__ x, float a, int64_t n)
{
    for (int64_t p = blockIdx.x * static_cast<int64_t>(kThr) + threadIdx.x; p < n;
         p += static_cast<int64_t>(gridDim.x) * kThr)
        y[p] = fmaf(a, x[p], y[p]);
}

gbst_status dense_dims(int64_t nx, int64_t ny, int64_t nz, DenseDims *d, const char *who)
{
    char msg[200];
    if (nx < 1 || ny < 1 || nz < 1 || nx > (1 << 30) || ny > (1 << 30) || nz > (1 << 30) ||
        nx * ny > (int64_t(1) << 40)) {
        snprintf(msg, sizeof msg, "%s: dims must be positive and at most 2^30 per axis", who);
        return record_error(GBST_EINVAL, msg);
    }
    d->nx = static_cast<int>(nx);
    d->ny = static_cast<int>(ny);
    d->nz = static_cast<int>(nz);
    return GBST_OK;
}

gbst_status launched(const char *who)
{
    const cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess)
        return GBST_OK;
    char msg[200];
    snprintf(msg, sizeof msg, "%s: %s", who, cudaGetErrorString(e));
    return record_error(GBST_ECUDA, msg);
}

}  // namespace

// Star stencil of radius r (weights w[0..r]) on a dense array; see k_star.
gbst_status dense_star(int r, const double *w, int64_t nx, int64_t ny, int64_t nz, const float *in, const float *pre,
                       const float *post, double alpha, bool accumulate, float *out, cudaStream_t s)
{
    DenseDims d;
    gbst_status st = dense_dims(nx, ny, nz, &d, "dense stencil");
    if (st != GBST_OK)
        return st;
    if (r < 1 || r > 4)
        return record_error(GBST_EINVAL, "dense stencil: radius must be 1..4");
    float wf[5] = {0, 0, 0, 0, 0};
    for (int m = 0; m <= r; ++m)
        wf[m] = static_cast<float>(w[m]);
    const float4 w03 = make_float4(wf[0], wf[1], wf[2], wf[3]);
    const int64_t n = nx * ny * nz;
    const int blocks = blocks_for_dense(n);
    const float a = static_cast<float>(alpha);
    const int acc = accumulate ? 1 : 0;
    switch (r) {
    case 1: k_star<1><<<dense_grid(d), kDX, 0, s>>>(d, in, pre, post, w03, wf[4], a, acc, out); break;
    case 2: k_star<2><<<dense_grid(d), kDX, 0, s>>>(d, in, pre, post, w03, wf[4], a, acc, out); break;
    case 3: k_star<3><<<dense_grid(d), kDX, 0, s>>>(d, in, pre, post, w03, wf[4], a, acc, out); break;
    default: k_star<4><<<dense_grid(d), kDX, 0, s>>>(d, in, pre, post, w03, wf[4], a, acc, out); break;
    }
    return launched("dense stencil");
}

namespace {
constexpr double kSixth[4] = {-20.0, 15.0, -6.0, 1.0};  // delta^6 per axis, w_0 .. w_3

FeatScales to_scales(const double *sc)
{
    FeatScales f;
    for (int k = 0; k < 8; ++k)
        f.s[k] = static_cast<float>(sc[k]);
    return f;
}
}  // namespace

// Closure input features (8 channels) from (u+, u^n, c_n) into x (channels-last BF16, 16
// channels, the last 8 zero): x_k = scales[k] f_k, see k_pack_features.  r, w: the star L.
// aux: also leave cn2, g_a, t5 and t6 in b (the transpose and closure_features_values read
// them); without it the two z-marching kernels compute the same x.  xch: channels per point
// of x, 16 (the last 8 zero) or, without aux, 8 (packed).
gbst_status closure_features_forward(const float *up, const float *un, const float *cn, int64_t nx, int64_t ny,
                                     int64_t nz, int r, const double *w, const double *scales,
                                     const ClosureFeatBufs &b, __nv_bfloat16 *x, bool aux, int xch, cudaStream_t s)
{
    DenseDims d;
    gbst_status st = dense_dims(nx, ny, nz, &d, "closure features");
    if (st != GBST_OK)
        return st;
    if (xch != 16 && (xch != 8 || aux))
        return record_error(GBST_EINVAL, "closure features: x has 16 channels per point, or 8 without aux");
    if (!aux) {
        // two z-marching launches: lu, then every channel (only b.lu is written besides x)
        if (r < 1 || r > 4)
            return record_error(GBST_EINVAL, "closure features: radius must be 1..4");
        float wf[5] = {0, 0, 0, 0, 0};
        for (int m = 0; m <= r; ++m)
            wf[m] = static_cast<float>(w[m]);
        const float4 w03 = make_float4(wf[0], wf[1], wf[2], wf[3]);
        const float4 w6 = make_float4(static_cast<float>(kSixth[0]), static_cast<float>(kSixth[1]),
                                      static_cast<float>(kSixth[2]), static_cast<float>(kSixth[3]));
        const FeatScales sc = to_scales(scales);
        const dim3 g = zmarch_grid(d), t(kFX, kFY);
        // four points per thread where rows and arrays allow 16-byte accesses
        const bool vec4 =
            d.nx % 4 == 0 && ((reinterpret_cast<uintptr_t>(un) | reinterpret_cast<uintptr_t>(b.lu)) & 15) == 0;
        if (vec4) {
            const dim3 g4((d.nx / 4 + kFX - 1) / kFX, g.y, g.z);
            switch (r) {
            case 1: k_lap4_z<1><<<g4, t, 0, s>>>(d, un, w03, wf[4], b.lu); break;
            case 2: k_lap4_z<2><<<g4, t, 0, s>>>(d, un, w03, wf[4], b.lu); break;
            case 3: k_lap4_z<3><<<g4, t, 0, s>>>(d, un, w03, wf[4], b.lu); break;
            default: k_lap4_z<4><<<g4, t, 0, s>>>(d, un, w03, wf[4], b.lu); break;
            }
        } else {
            switch (r) {
            case 1: k_lap_z<1><<<g, t, 0, s>>>(d, un, w03, wf[4], b.lu); break;
            case 2: k_lap_z<2><<<g, t, 0, s>>>(d, un, w03, wf[4], b.lu); break;
            case 3: k_lap_z<3><<<g, t, 0, s>>>(d, un, w03, wf[4], b.lu); break;
            default: k_lap_z<4><<<g, t, 0, s>>>(d, un, w03, wf[4], b.lu); break;
            }
        }
        if ((st = launched("closure features")) != GBST_OK)
            return st;
        if (xch == 8) {
            switch (r) {
            case 1: k_features_z<1, 8><<<g, t, 0, s>>>(d, up, un, cn, b.lu, w03, wf[4], w6, sc, x); break;
            case 2: k_features_z<2, 8><<<g, t, 0, s>>>(d, up, un, cn, b.lu, w03, wf[4], w6, sc, x); break;
            case 3: k_features_z<3, 8><<<g, t, 0, s>>>(d, up, un, cn, b.lu, w03, wf[4], w6, sc, x); break;
            default: k_features_z<4, 8><<<g, t, 0, s>>>(d, up, un, cn, b.lu, w03, wf[4], w6, sc, x); break;
            }
        } else {
            switch (r) {
            case 1: k_features_z<1, 16><<<g, t, 0, s>>>(d, up, un, cn, b.lu, w03, wf[4], w6, sc, x); break;
            case 2: k_features_z<2, 16><<<g, t, 0, s>>>(d, up, un, cn, b.lu, w03, wf[4], w6, sc, x); break;
            case 3: k_features_z<3, 16><<<g, t, 0, s>>>(d, up, un, cn, b.lu, w03, wf[4], w6, sc, x); break;
            default: k_features_z<4, 16><<<g, t, 0, s>>>(d, up, un, cn, b.lu, w03, wf[4], w6, sc, x); break;
            }
        }
        return launched("closure features");
    }
    k_cn2_grads<<<dense_grid(d), kDX, 0, s>>>(d, cn, b.cn2, b.g[0], b.g[1], b.g[2]);
    if ((st = launched("closure features")) != GBST_OK)
        return st;
    if ((st = dense_star(r, w, nx, ny, nz, un, nullptr, nullptr, 1.0, false, b.lu, s)) != GBST_OK)
        return st;
    if ((st = dense_star(r, w, nx, ny, nz, b.lu, b.cn2, b.cn2, 1.0, false, b.t5, s)) != GBST_OK)
        return st;
    if ((st = dense_star(3, kSixth, nx, ny, nz, un, nullptr, b.cn2, 1.0, false, b.t6, s)) != GBST_OK)
        return st;
    k_pack_features<<<dense_grid(d), kDX, 0, s>>>(d, up, un, b.cn2, b.t6, b.t5, b.lu, b.g[0], b.g[1], b.g[2],
                                            to_scales(scales), x);
    return launched("closure features");
}

// Transpose of closure_features_forward (which must have run for the same c_n, so that
// b.cn2 and b.g hold its values): from the cotangent dx of x, g_up and g_un are written.
gbst_status closure_features_adjoint(const __nv_bfloat16 *dx, int64_t nx, int64_t ny, int64_t nz, int r,
                                     const double *w, const double *scales, const ClosureFeatBufs &b, float *g_up,
                                     float *g_un, cudaStream_t s)
{
    DenseDims d;
    gbst_status st = dense_dims(nx, ny, nz, &d, "closure feature adjoint");
    if (st != GBST_OK)
        return st;
    const int blocks = blocks_for_dense(nx * ny * nz);
    float *e4 = b.t6, *e5 = b.t5, *e6 = b.lu, *e7 = b.e7;
    k_unpack_features_adj<<<blocks, kThr, 0, s>>>(d, dx, b.cn2, b.g[0], b.g[1], b.g[2], to_scales(scales), g_up,
                                                  g_un, e4, e5, e6, e7);
    if ((st = launched("closure feature adjoint")) != GBST_OK)
        return st;
    if ((st = dense_star(3, kSixth, nx, ny, nz, e4, nullptr, nullptr, 1.0, true, g_un, s)) != GBST_OK)
        return st;
    if ((st = dense_star(r, w, nx, ny, nz, e5, nullptr, nullptr, 1.0, false, b.tmp, s)) != GBST_OK)
        return st;
    if ((st = dense_star(r, w, nx, ny, nz, b.tmp, b.cn2, nullptr, 1.0, true, g_un, s)) != GBST_OK)
        return st;
    k_div_acc<<<dense_grid(d), kDX, 0, s>>>(d, e6, b.g[0], b.g[1], b.g[2], -1.0f, g_un);
    if ((st = launched("closure feature adjoint")) != GBST_OK)
        return st;
    return dense_star(r, w, nx, ny, nz, e7, nullptr, nullptr, 1.0, true, g_un, s);
}

// The unscaled FP32 features f_0 .. f_7, channel-major (out + k * n), after
// closure_features_forward has filled b for the same inputs.
gbst_status closure_features_values(const float *up, const float *un, int64_t nx, int64_t ny, int64_t nz,
                                    const ClosureFeatBufs &b, float *out, cudaStream_t s)
{
    DenseDims d;
    gbst_status st = dense_dims(nx, ny, nz, &d, "closure feature values");
    if (st != GBST_OK)
        return st;
    k_feature_values<<<dense_grid(d), kDX, 0, s>>>(d, up, un, b.cn2, b.t6, b.t5, b.lu, b.g[0],
                                                                    b.g[1], b.g[2], out);
    return launched("closure feature values");
}

gbst_status rollout_sums(const float *u, const float *ref, int64_t n, double *sums, cudaStream_t s)
{
    k_roll_sums<<<std::min(blocks_for_dense(n), 4096), kThr, 0, s>>>(u, ref, n, sums);
    return launched("rollout loss");
}

gbst_status rollout_grad(float *u, const float *ref, int64_t n, const double *sums, double scale, cudaStream_t s)
{
    k_roll_grad<<<blocks_for_dense(n), kThr, 0, s>>>(u, ref, n, sums, scale);
    return launched("rollout loss gradient");
}

gbst_status dense_axpy(float *y, const float *x, float a, int64_t n, cudaStream_t s)
{
    k_axpy<<<blocks_for_dense(n), kThr, 0, s>>>(y, x, a, n);
    return launched("dense axpy");
}

}  // namespace gbst

using namespace gbst;

extern "C" gbst_status stencil_wave_adjoint_dense(int space_order, int64_t nx, int64_t ny, int64_t nz,
                                                  const float *kappa, const float *lam_next, float *lam_cur,
                                                  float *lam_prev, void *stream)
{
    static const char *who = "stencil_wave_adjoint_dense";
    if (!kappa || !lam_next || !lam_cur)
        return record_error(GBST_EINVAL, "stencil_wave_adjoint_dense: null kappa, lam_next or lam_cur");
    if (space_order != 2 && space_order != 4 && space_order != 8)
        return record_error(GBST_EINVAL, "stencil_wave_adjoint_dense: space_order must be 2, 4 or 8");
    DenseDims d;
    gbst_status st = dense_dims(nx, ny, nz, &d, who);
    if (st != GBST_OK)
        return st;
    double w[9];
    st = stencil_fd_weights(space_order, w);
    if (st != GBST_OK)
        return st;
    float wf[5] = {0, 0, 0, 0, 0};
    for (int m = 0; m <= space_order / 2; ++m)
        wf[m] = static_cast<float>(w[m]);
    const float4 w03 = make_float4(wf[0], wf[1], wf[2], wf[3]);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int blocks = blocks_for_dense(nx * ny * nz);
    switch (space_order) {
    case 2: k_wave_adjoint<1><<<dense_grid(d), kDX, 0, s>>>(d, kappa, lam_next, w03, wf[4], lam_cur, lam_prev); break;
    case 4: k_wave_adjoint<2><<<dense_grid(d), kDX, 0, s>>>(d, kappa, lam_next, w03, wf[4], lam_cur, lam_prev); break;
    default: k_wave_adjoint<4><<<dense_grid(d), kDX, 0, s>>>(d, kappa, lam_next, w03, wf[4], lam_cur, lam_prev); break;
    }
    return launched(who);
}
