// Temporally blocked streaming heat sweep (two forward-Euler steps per pass
// over HBM), FP32 storage, 3D, zero Dirichlet ghosts.
//
// The step-1 field u' = u + a L(u) is computed on the output tile grown by r
// in y and by one 16-byte chunk (4 points >= r) in x, from input planes that
// carry a 2r halo; u' is kept on chip (a ring of shared-memory planes for its
// x/y neighbours, a register queue for its z neighbours) and the step-2 field
// u'' = u' + a L(u') is computed on the tile and stored.  Points of u' outside
// the interior are zero, as the ghost cells of a stored u' would be, and every
// point is updated with the same arithmetic, in the same order, as the
// single-step kernel, so a blocked run equals the same number of single steps
// bit for bit.  Overlapped tiles recompute the u' halo instead of exchanging
// it (overlapped temporal blocking; the paper's related work, Section 7).
//
// CTA: NW "main" warps (warp w owns rows w*PY .. w*PY+PY-1 of the grown tile,
// lane l owns x chunk l), one "edge" warp (the two x-halo chunks of every row
// group, step 1 only) and one TMA producer warp.  Input planes arrive as in the
// single-step kernel: ring of S = r + 1 + D slots, full/empty mbarrier pairs.
// Per u' plane buffer an mbarrier (one arrival per consumer warp; waits are
// bounded like all others) orders the plane's writes before its step-2 reads;
// step 2 runs one plane behind step 1, so that wait is usually already met.  A launch with a.tb_single = 1 performs only step 1 (the odd step of
// a run) and stores it.
#pragma once
#include <type_traits>

#include "sweep_stream.cuh"

namespace gbst {
namespace sweep {
namespace {

__device__ __forceinline__ void sts128(unsigned char *p, const uint4 &v)
{
    *reinterpret_cast<uint4 *>(p) = v;
}

// f(integral_constant<int, 0>), ..., f(integral_constant<int, N-1>) while f returns true.
template <int N, int I = 0, class F>
__device__ __forceinline__ bool static_for(F &f)
{
    if constexpr (I < N) {
        if (!f(std::integral_constant<int, I>{}))
            return false;
        return static_for<N, I + 1>(f);
    } else {
        return true;
    }
}

template <int R, int NW, int PY, int D>
struct TbShape {
    static constexpr int PX = 4;                     // FP32 points per 16-byte chunk
    static constexpr int TX = 32 * PX;               // tile width (points)
    static constexpr int TY = NW * PY - 2 * R;       // tile height (rows)
    static constexpr int IN_W = TX + 4 * PX;         // input box width: tile + 2 chunks per side
    static constexpr int IN_H = TY + 4 * R;          // input box height: tile + 2r per side
    static constexpr int U_W = TX + 2 * PX;          // u' plane width: tile + 1 chunk per side
    static constexpr int U_H = TY + 2 * R;           // u' plane height
    static constexpr int U_BYTES = (U_W * U_H * 4 + 127) / 128 * 128;
    static constexpr int NU = R + 2;                 // u' planes kept
    static constexpr int QN = 2 * R + 1;             // z-queue length
    static constexpr int S = R + 1 + D;              // input plane slots
    static constexpr int NB = D + 1;                 // mbarrier pairs
    static constexpr int PAD = (R * U_W * 4 + 127) / 128 * 128;  // rows read past the last u' plane
    static_assert(TY >= 1, "tile height");
    static_assert(2 * NW <= 32, "the edge warp covers both x-halo chunks of every row group");
    static_assert(R <= PX, "x halo chunk must cover the radius");
};

// One star-stencil heat update of PY rows x 4 FP32 points, in the single-step
// kernel's order: own values from queue slot QC of q, x/y neighbours from
// shared memory at `cb` (row pitch `row` bytes), z neighbours from queue slots
// QC -+ m.  (Taking the x neighbours from adjacent lanes by shuffles, with the
// tile-edge lanes reading shared memory -- by a branch or by predicated loads --
// measured 4-23 % slower for order 2.)
template <int R, int PY, int QC, bool SX>
__device__ __forceinline__ void tb_update(const float2 (&q)[2 * R + 1][PY][2], const unsigned char *cb,
                                          const int row, const float2 wc2, const float2 (&w2)[R + 1],
                                          const float2 a2, float (&o)[PY][4])
{
    using St = Storage<GBST_F32>;
    constexpr int PX = 4, PP = 2, QN = 2 * R + 1;
    uint4 ylo[R], yhi[R], xl[PY], xr[PY];
#pragma unroll
    for (int m = 1; m <= R; ++m) {
        ylo[m - 1] = lds128(cb - m * row);
        yhi[m - 1] = lds128(cb + (PY - 1 + m) * row);
    }
#pragma unroll
    for (int r_ = 0; r_ < PY; ++r_) {
        xl[r_] = load_left<GBST_F32, R>(cb + r_ * row - 16);
        xr[r_] = load_right<GBST_F32, R>(cb + r_ * row + 16);
    }
    auto xel = [&](int r_, int e) -> float {
        if (e < 0)
            return St::get(xl[r_], PX + e);
        if (e >= PX)
            return St::get(xr[r_], e - PX);
        return (e & 1) ? q[QC][r_][e >> 1].y : q[QC][r_][e >> 1].x;
    };
    auto yrow = [&](int rr, int pp) -> float2 {
        if (rr < 0)
            return St::pair(ylo[-rr - 1], pp);
        if (rr >= PY)
            return St::pair(yhi[rr - PY], pp);
        return q[QC][rr][pp];
    };
    float2 sv[PY][PP];
#pragma unroll
    for (int r_ = 0; r_ < PY; ++r_)
#pragma unroll
        for (int pp = 0; pp < PP; ++pp)
            sv[r_][pp] = __fmul2_rn(wc2, q[QC][r_][pp]);
#pragma unroll
    for (int m = 1; m <= R; ++m) {
#pragma unroll
        for (int r_ = 0; r_ < PY; ++r_) {
#pragma unroll
            for (int pp = 0; pp < PP; ++pp) {
                const int e = 2 * pp;
                const float2 xm = make_float2(xel(r_, e - m), xel(r_, e + 1 - m));
                const float2 xp = make_float2(xel(r_, e + m), xel(r_, e + 1 + m));
                float2 xs;
                if (SX && (m & 1)) {  // operands straddle the packed pairs: two scalar additions
                    xs.x = __fadd_rn(xm.x, xp.x);
                    xs.y = __fadd_rn(xm.y, xp.y);
                } else {
                    xs = __fadd2_rn(xm, xp);
                }
                float2 t = __fadd2_rn(xs, __fadd2_rn(yrow(r_ - m, pp), yrow(r_ + m, pp)));
                t = __fadd2_rn(t, __fadd2_rn(q[(QC - m + 2 * QN) % QN][r_][pp], q[(QC + m) % QN][r_][pp]));
                sv[r_][pp] = __ffma2_rn(w2[m], t, sv[r_][pp]);
            }
        }
    }
#pragma unroll
    for (int r_ = 0; r_ < PY; ++r_)
#pragma unroll
        for (int pp = 0; pp < PP; ++pp) {
            const float2 ov = __ffma2_rn(a2, sv[r_][pp], q[QC][r_][pp]);
            o[r_][2 * pp] = ov.x;
            o[r_][2 * pp + 1] = ov.y;
        }
}

template <int R, int NW, int PY, int D, int MINB, int OPT = 0>
__global__ void __launch_bounds__((NW + 2) * 32, MINB) k_tb(const SweepArgs a, const int slot_bytes)
{
    using Sh = TbShape<R, NW, PY, D>;
    using St = Storage<GBST_F32>;
    constexpr int PX = Sh::PX, TX = Sh::TX, TY = Sh::TY;
    constexpr int QN = Sh::QN, S = Sh::S, NB = Sh::NB, NU = Sh::NU;
    constexpr int IN_ROW = Sh::IN_W * 4, U_ROW = Sh::U_W * 4;
    constexpr int PP = PX / 2;
    static_assert((2 * NB + NU + 1) * 8 + 8 + 4 * NB <= 256, "barrier header");

    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *full = reinterpret_cast<uint64_t *>(smem);
    uint64_t *empty = full + NB;
    uint64_t *ubar = empty + NB;  // per u' plane buffer: plane written (one arrival per consumer warp)
    uint64_t *uend = ubar + NU;   // end of a unit: every consumer warp is done with the u' planes
    volatile int *abort_flag = reinterpret_cast<volatile int *>(uend + 1);
    // unit of a unit's first iteration, by barrier pair (-1: no more units), as in k_stream
    volatile int *uidx = reinterpret_cast<volatile int *>(smem + (2 * NB + NU + 1) * 8 + 8);
    unsigned char *slots = smem + 256;
    unsigned char *ubuf = slots + S * slot_bytes;  // NU u' planes of Sh::U_BYTES

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            mbar_init(&full[b], 1);
            mbar_init(&empty[b], NW + 1);
        }
#pragma unroll
        for (int b = 0; b < NU; ++b)
            mbar_init(&ubar[b], NW + 1);
        mbar_init(uend, NW + 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    const int parity = a.parity;
    const bool single = a.tb_single != 0;

    // ------------------------------------------------------------ producer
    if (warp == NW + 1) {
        if (lane != 0)
            return;
        int it = 0;
        for (int ui = first_unit(a); ui < a.nunits; ui = next_unit(a, ui)) {
            const Unit u = a.units[ui];
            const GridDev &g = a.grids[u.grid];
            const int bx = (u.tile % g.tiles_x) * TX, by = (u.tile / g.tiles_x) * TY;
            const CUtensorMap *map = &g.tmap_tb[parity];  // every ghost row and plane of the layout
            const uint32_t bytes = static_cast<uint32_t>(g.box_bytes);
            const int L = (u.z1 - u.z0) + 4 * R + (single ? 0 : 1);
            const int gs = g.ghost - 2 * R;  // map coordinate of interior row / plane 0, less 2r
            for (int l = 0; l < L; ++l, ++it) {
                if (it >= NB && !wait_or_abort(&empty[it % NB], ((it / NB) - 1) & 1, abort_flag))
                    goto drain;
                if (l == 0)
                    uidx[it % NB] = ui;  // published by the arrive below
                mbar_arrive_expect_tx(&full[it % NB], bytes);
                // map coordinates: x from bx - 2 chunks (the map starts one chunk before the
                // interior), y from by - 2r, plane z0 - 2r + l (the map starts `ghost` rows
                // and planes before the interior); outside the tensor the load fills zeros
                tma_load_plane(slots + (it % S) * slot_bytes, map, &full[it % NB], bx - PX, by + gs,
                               u.z0 + gs + l);
            }
        }
        // sentinel iteration: no more units
        if (it >= NB && !wait_or_abort(&empty[it % NB], ((it / NB) - 1) & 1, abort_flag))
            goto drain;
        uidx[it % NB] = -1;
        mbar_arrive(&full[it % NB]);
        ++it;
        units_done(a);
    drain:
        if (*abort_flag) {
            atomicCAS(a.err, 0, static_cast<int>(kDevTimeoutTma));
            for (int k = it - NB < 0 ? 0 : it - NB; k < it; ++k) {
                const unsigned long long t0 = global_ns();
                while (!mbar_try_wait(&full[k % NB], (k / NB) & 1) && global_ns() - t0 < 50000000ull) {
                }
            }
        }
        return;
    }

    // ----------------------------------------------------------- consumers
    const bool is_edge = warp == NW;
    // edge lanes: e < NW left chunk of row group e, NW <= e < 2 NW right chunk of group e - NW
    const bool active = !is_edge || lane < 2 * NW;
    const int grp = is_edge ? (lane < NW ? lane : (active ? lane - NW : 0)) : warp;
    const int cx = is_edge ? (lane < NW || !active ? -PX : TX) : lane * PX;  // chunk x offset in the tile
    const int rho0 = grp * PY;                                     // first row of the grown tile
    // step-2 rows of this main warp (grown-tile rows [r, TY + r))
    bool s2row[PY];
    bool any_s2 = false;
#pragma unroll
    for (int k = 0; k < PY; ++k) {
        s2row[k] = !is_edge && rho0 + k >= R && rho0 + k < TY + R;
        any_s2 = any_s2 || s2row[k];
    }
    const float2 wc2 = make_float2(a.wc, a.wc);
    float2 w2[R + 1];
#pragma unroll
    for (int m = 1; m <= R; ++m)
        w2[m] = make_float2(a.w[m], a.w[m]);
    const int in_off = (rho0 + R) * IN_ROW + (cx + 2 * PX) * 4;
    const int u_off = rho0 * U_ROW + (cx + PX) * 4;

    float2 q1[QN][PY][PP];  // input u, own points, by plane index mod QN
    float2 q2[QN][PY][PP];  // u', own points, by u' plane index mod QN
    int slot_n = 0, bar_i = 0;  // ring slot, barrier pair
    uint32_t par = 0, upar = 0; // phase parities of full/empty and of uend
    // u' planes written so far by this CTA, pc, kept as its buffer uw = pc mod NU
    // and the phase parity uwp = (pc / NU) & 1 of that buffer's barrier
    int uw = 0;
    uint32_t uwp = 0;
    auto advance = [&]() {
        slot_n = slot_n + 1 == S ? 0 : slot_n + 1;
        if (++bar_i == NB) {
            bar_i = 0;
            par ^= 1;
        }
    };

    for (;;) {
        // the first iteration of the next unit, or the sentinel
        if (!wait_or_abort(&full[bar_i], par, abort_flag)) {
            atomicCAS(a.err, 0, static_cast<int>(kDevTimeoutTma));
            return;
        }
        const int ui = uidx[bar_i];
        if (ui < 0) {
            __syncwarp();
            if (lane == 0)
                mbar_arrive(&empty[bar_i]);
            return;
        }
        const Unit u = a.units[ui];
        const GridDev *gp = a.grids + u.grid;
        const int tiles_x = gp->tiles_x;
        const int64_t nx = gp->nx, ny = gp->ny, nz = gp->nz;
        const int64_t pitch = gp->pitch, rows = gp->rows, origin = gp->origin;
        unsigned char *__restrict__ outbase = static_cast<unsigned char *>(gp->buf[1 - parity]);
        const float2 a2 = make_float2(gp->heat_a, gp->heat_a);
        const int bx = (u.tile % tiles_x) * TX, by = (u.tile / tiles_x) * TY;
        // Masks of this thread's u' points: u' is zero outside the global domain (the
        // ghost cells of a stored u' would be); across a face shared with another
        // subdomain the ghost region holds that subdomain's u (two-step exchange) and
        // u' there is the value the neighbour computes itself.  Stores: interior only.
        const int fi = gp->face_int;
        const int64_t xlo = (fi & 1) ? -(1ll << 40) : 0, xhi = (fi & 2) ? (1ll << 40) : nx;
        const int64_t ylo = (fi & 4) ? -(1ll << 40) : 0, yhi = (fi & 8) ? (1ll << 40) : ny;
        const int zlo = (fi & 16) ? -(1 << 30) : 0, zhi = (fi & 32) ? (1 << 30) : static_cast<int>(nz);
        bool yin[PY], ysto[PY];
#pragma unroll
        for (int k = 0; k < PY; ++k) {
            const int64_t y = static_cast<int64_t>(by) - R + rho0 + k;
            yin[k] = y >= ylo && y < yhi;
            ysto[k] = y >= 0 && y < ny;
        }
        bool xin[PX], xsto[PX];
#pragma unroll
        for (int i = 0; i < PX; ++i) {
            const int64_t x = static_cast<int64_t>(bx) + cx + i;
            xin[i] = x >= xlo && x < xhi;
            xsto[i] = x >= 0 && x < nx;
        }
        // every u' point of this thread lies inside the grid in x and y (the usual
        // case): only planes outside [0, nz) need zeroing
        bool inner = true;
#pragma unroll
        for (int k = 0; k < PY; ++k)
            inner = inner && yin[k];
#pragma unroll
        for (int i = 0; i < PX; ++i)
            inner = inner && xin[i];
        const bool xfull = bx + cx + PX <= nx;
        bool st_row[PY];  // rows this thread stores (step-2 rows, or step-1 rows in single mode)
#pragma unroll
        for (int k = 0; k < PY; ++k)
            st_row[k] = s2row[k] && ysto[k] && bx + cx < nx;
        const int64_t plane_elems = rows * pitch;
        const int64_t row_stride = pitch * 4;
        const int64_t plane_bytes = plane_elems * 4;
        // output pointer at plane z0, grown-tile row rho0 (y = by - r + rho0), column bx + cx
        unsigned char *optr = outbase +
                              (origin + (static_cast<int64_t>(u.z0) * rows + (by - R + rho0)) * pitch + bx + cx) * 4;
        int64_t o2off = 0;  // byte offset of the next step-2 output plane from optr

        const int nout = u.z1 - u.z0;
        // input planes of the unit; two-step mode takes one more so that the last
        // output plane's step 2 (one plane behind step 1) runs inside the loop
        const int L = nout + 4 * R + (single ? 0 : 1);
        int j0 = 0;
        // Iteration j = j0 + k of the z-march (k is a compile-time constant, so every
        // queue slot below is one too): step 2 on u' plane P - 1 - r, then step 1 on
        // input plane j - r giving u' plane P = j - 2r.  Step 2 waits for plane P - 1,
        // which every consumer warp finished one iteration earlier (split-phase
        // barrier), and reads its u' z-neighbours before step 1 overwrites the
        // oldest queue slot.  Returns false when a wait gave up.
        auto body = [&](auto kc) -> bool {
            constexpr int k = decltype(kc)::value;
            const int j = j0 + k;
            if (j >= L)
                return true;
            if (!wait_or_abort(&full[bar_i], par, abort_flag))
                return false;
            // newest input plane into the z-queue
            {
                const unsigned char *nb = slots + slot_n * slot_bytes + in_off;
#pragma unroll
                for (int r_ = 0; r_ < PY; ++r_) {
                    const uint4 v = lds128(nb + r_ * IN_ROW);
#pragma unroll
                    for (int pp = 0; pp < PP; ++pp)
                        q1[k][r_][pp] = St::pair(v, pp);
                }
            }
            if (!single && j >= 4 * R + 1) {
                // u' plane P - 1 (count pc - 1: buffer uw - 1 mod NU) is complete in shared memory
                const int up = uw == 0 ? NU - 1 : uw - 1;
                if (!wait_or_abort(&ubar[up], uw == 0 ? uwp ^ 1u : uwp, abort_flag))
                    return false;
                unsigned char *op = optr + o2off;
                o2off += plane_bytes;
                if (any_s2) {
                    // step 2 on u' plane P - 1 - r = output plane z0 + j - 4r - 1, in
                    // buffer (pc - 1 - r) mod NU = (uw + 1) mod NU since NU = r + 2
                    static_assert(NU == R + 2, "u' ring length");
                    constexpr int qc2 = (k - 3 * R - 1 + 4 * QN) % QN;
                    float o[PY][PX];
                    tb_update<R, PY, qc2, (OPT & kOptScalarOddX) != 0>(q2, ubuf + (uw + 1 == NU ? 0 : uw + 1) * Sh::U_BYTES + u_off, U_ROW,
                                          wc2, w2, a2, o);
#pragma unroll
                    for (int r_ = 0; r_ < PY; ++r_) {
                        if (st_row[r_]) {
                            if (xfull) {
                                *reinterpret_cast<uint4 *>(op + r_ * row_stride) = St::pack(o[r_]);
                            } else {
#pragma unroll
                                for (int i = 0; i < PX; ++i)
                                    if (xsto[i])
                                        St::store1(op + r_ * row_stride + i * 4, o[r_][i]);
                            }
                        }
                    }
                }
            }
            const bool s1 = j >= 2 * R;  // step 1 on input plane j - r (u' plane P = j - 2r)
            if (s1 && active) {
                constexpr int qc1 = (k - R + QN) % QN;
                const int slot_c = slot_n >= R ? slot_n - R : slot_n - R + S;
                float o[PY][PX];
                tb_update<R, PY, qc1, (OPT & kOptScalarOddX) != 0>(q1, slots + slot_c * slot_bytes + in_off, IN_ROW, wc2, w2, a2, o);
                // u' plane index (interior z) of this result; u' is zero outside the interior
                const int zq = u.z0 - 3 * R + j;
                if (zq < zlo || zq >= zhi) {
#pragma unroll
                    for (int r_ = 0; r_ < PY; ++r_)
#pragma unroll
                        for (int i = 0; i < PX; ++i)
                            o[r_][i] = 0.0f;
                } else if (!inner) {
#pragma unroll
                    for (int r_ = 0; r_ < PY; ++r_)
#pragma unroll
                        for (int i = 0; i < PX; ++i)
                            if (!(yin[r_] && xin[i]))
                                o[r_][i] = 0.0f;
                }
                if (single) {
                    // one step only: store u' of planes [z0, z1)
                    if (zq >= u.z0 && zq < u.z1) {
                        unsigned char *op = optr + static_cast<int64_t>(zq - u.z0) * plane_bytes;
#pragma unroll
                        for (int r_ = 0; r_ < PY; ++r_) {
                            if (st_row[r_]) {
                                if (xfull) {
                                    *reinterpret_cast<uint4 *>(op + r_ * row_stride) = St::pack(o[r_]);
                                } else {
#pragma unroll
                                    for (int i = 0; i < PX; ++i)
                                        if (xsto[i])
                                            St::store1(op + r_ * row_stride + i * 4, o[r_][i]);
                                }
                            }
                        }
                    }
                } else {
                    constexpr int qn2 = (k - 2 * R + 2 * QN) % QN;
                    unsigned char *ub = ubuf + uw * Sh::U_BYTES + u_off;
#pragma unroll
                    for (int r_ = 0; r_ < PY; ++r_) {
#pragma unroll
                        for (int pp = 0; pp < PP; ++pp)
                            q2[qn2][r_][pp] = make_float2(o[r_][2 * pp], o[r_][2 * pp + 1]);
                        sts128(ub + r_ * U_ROW, St::pack(o[r_]));
                    }
                }
            }
            // the input planes of this iteration are no longer read; u' plane P is written
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(&empty[bar_i]);
                if (s1 && !single)
                    mbar_arrive(&ubar[uw]);
            }
            if (s1 && !single && ++uw == NU) {
                uw = 0;
                uwp ^= 1u;
            }
            advance();
            return true;
        };
        bool ok = true;
        for (; j0 < L && ok; j0 += QN)
            ok = static_for<QN>(body);
        // all u' reads of this unit are done before the next unit overwrites the planes
        if (ok && !single) {
            __syncwarp();
            if (lane == 0)
                mbar_arrive(uend);
            ok = wait_or_abort(uend, upar, abort_flag);
            upar ^= 1;
        }
        if (!ok) {
            // a wait gave up (the producer may have left already): report it here
            atomicCAS(a.err, 0, static_cast<int>(kDevTimeoutTma));
            return;
        }
    }
}

}  // namespace

template <int R, int NW, int PY, int D, int MINB, int OPT = 0>
constexpr Entry tb_entry()
{
    return Entry{StreamVariant{R, GBST_HEAT, GBST_F32, true, (NW + 1) * 32, PY, D, MINB, 32, 2, false, 1, OPT},
                 &k_tb<R, NW, PY, D, MINB, OPT>};
}

}  // namespace sweep
}  // namespace gbst
