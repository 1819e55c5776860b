// Fused multi-field sweep (several stencils in one pass over memory): a system
// of NF FP32 fields on one 3D grid with zero ghosts,
//     u_k^{n+1} = u_k^n + sum_j A[k][j] L(u_j^n),   k = 0 .. NF-1,
// a synthetic stand-in for the paper's multi-stencil regions (Section 6.2,
// several stencils fused into one loop nest).  One pass reads each field once
// and writes each once; L(u_j) is computed once per point and used by every
// output (unfused, each output would read every field it depends on).
//
// The CTA is the single-step streaming kernel's (TMA producer warp, plane ring
// with full/empty mbarrier pairs, register z-queues), with NF boxes per ring
// slot, one per field, completing on the same mbarrier.  Each L(u_j) is summed
// in the single-step kernel's order, then o_k = u_k, o_k = fma(A[k][j], L_j, o_k)
// for j = 0 .. NF-1; with A = a I the result equals NF heat sweeps bit for bit.
// The fields are NF consecutive grids of a batch handle (same layout).
#pragma once
#include "sweep_stream.cuh"

namespace gbst {
namespace sweep {
namespace {

template <int R, int NF, int NC, int PY, int D, int MINB, int TXT>
__global__ void __launch_bounds__((NC + 1) * 32, MINB) k_system(const SweepArgs a, const int slot_bytes)
{
    using St = Storage<GBST_F32>;
    constexpr int NT = NC * 32;
    constexpr int PX = St::PX, ES = St::ES, G = PX, PP = PX / 2;
    constexpr int QN = 2 * R + 1;
    constexpr int S = R + 1 + D;
    constexpr int NB = D + 1;
    constexpr int TX = TXT * PX;
    constexpr int TY = (NT / TXT) * PY;
    constexpr int ROW_BYTES = (TX + 2 * G) * ES;
    static_assert(R <= G, "x halo must cover the radius");
    static_assert(2 * NB * 8 + 16 + 4 * NB <= 256, "barrier header");
    static_assert(NF >= 2 && NF <= 4, "2 to 4 fields");

    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *full = reinterpret_cast<uint64_t *>(smem);
    uint64_t *empty = full + NB;
    volatile int *abort_flag = reinterpret_cast<volatile int *>(empty + NB);
    volatile int *uidx = reinterpret_cast<volatile int *>(smem + 2 * NB * 8 + 16);  // as in k_stream
    unsigned char *slots = smem + 256;  // slot s, field f: slots + (s * NF + f) * slot_bytes

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
    const int parity = a.parity;

    if (warp == NC) {
        // ---------------------------------------------------------- producer
        if (lane != 0)
            return;
        int it = 0;
        bool ok = true;
        for (int ui = first_unit(a); ui < a.nunits && ok; ui = next_unit(a, ui)) {
            const Unit u = a.units[ui];
            const GridDev &g0 = a.grids[u.grid];
            const int bx = (u.tile % g0.tiles_x) * TX, by = (u.tile / g0.tiles_x) * TY;
            const uint32_t bytes = static_cast<uint32_t>(g0.box_bytes);
            const int L = (u.z1 - u.z0) + 2 * R;
            for (int l = 0; l < L; ++l, ++it) {
                if (it >= NB && !wait_or_abort(&empty[it % NB], ((it / NB) - 1) & 1, abort_flag)) {
                    ok = false;
                    break;
                }
                if (l == 0)
                    uidx[it % NB] = ui;  // published by the arrive below
                uint64_t *bar = &full[it % NB];
                mbar_arrive_expect_tx(bar, bytes * NF);
#pragma unroll
                for (int f = 0; f < NF; ++f)
                    tma_load_plane(slots + ((it % S) * NF + f) * slot_bytes, &a.grids[u.grid + f].tmap[parity], bar,
                                   bx, by, u.z0 + l);
            }
        }
        // sentinel iteration: no more units
        if (ok && it >= NB && !wait_or_abort(&empty[it % NB], ((it / NB) - 1) & 1, abort_flag))
            ok = false;
        if (ok) {
            uidx[it % NB] = -1;
            mbar_arrive(&full[it % NB]);
            ++it;
            units_done(a);
        }
        if (!ok) {
            atomicCAS(a.err, 0, static_cast<int>(kDevTimeoutTma));
            for (int k = it - NB < 0 ? 0 : it - NB; k < it; ++k) {
                const unsigned long long t0 = global_ns();
                while (!mbar_try_wait(&full[k % NB], (k / NB) & 1) && global_ns() - t0 < 50000000ull) {
                }
            }
        }
        return;
    }

    // ------------------------------------------------------------- consumers
    const int tid = threadIdx.x;
    float2 q[NF][QN][PY][PP];
    int slot_n = 0, bar_i = 0;
    uint32_t par = 0;
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
    float2 A2[NF][NF];
#pragma unroll
    for (int k = 0; k < NF; ++k)
#pragma unroll
        for (int j = 0; j < NF; ++j)
            A2[k][j] = make_float2(a.coupling[k * NF + j], a.coupling[k * NF + j]);

    bool ok = true;
    while (ok) {
        // the first iteration of the next unit, or the sentinel
        if (!wait_or_abort(&full[bar_i], par, abort_flag)) {
            ok = false;
            break;
        }
        const int ui = uidx[bar_i];
        if (ui < 0) {
            __syncwarp();
            if (lane == 0)
                mbar_arrive(&empty[bar_i]);
            advance();
            break;
        }
        const Unit u = a.units[ui];
        const GridDev *gp = a.grids + u.grid;
        const int tiles_x = gp->tiles_x;
        const int64_t nx = gp->nx, ny = gp->ny;
        const int64_t pitch = gp->pitch, rows = gp->rows, origin = gp->origin;
        unsigned char *outb[NF];
#pragma unroll
        for (int f = 0; f < NF; ++f)
            outb[f] = static_cast<unsigned char *>(gp[f].buf[1 - parity]);
        const int tx = tid % TXT, ty = tid / TXT;
        const int x0 = (u.tile % tiles_x) * TX + tx * PX;
        const int y0 = (u.tile / tiles_x) * TY + ty * PY;
        const int own_off = (R + ty * PY) * ROW_BYTES + (G + tx * PX) * ES;
        const bool xfull = x0 + PX <= nx;
        bool row_ok[PY];
#pragma unroll
        for (int r_ = 0; r_ < PY; ++r_)
            row_ok[r_] = y0 + r_ < ny && x0 < nx;
        const int64_t plane_bytes = rows * pitch * ES;
        const int64_t row_stride = pitch * ES;
        int64_t ooff = (origin + (static_cast<int64_t>(u.z0) * rows + y0) * pitch + x0) * ES;

        auto load_newest = [&](float2 (&qq)[NF][QN][PY][PP], const int qs) {
#pragma unroll
            for (int f = 0; f < NF; ++f) {
                const unsigned char *nb = slots + (slot_n * NF + f) * slot_bytes + own_off;
#pragma unroll
                for (int r_ = 0; r_ < PY; ++r_) {
                    const uint4 v = lds128(nb + r_ * ROW_BYTES);
#pragma unroll
                    for (int pp = 0; pp < PP; ++pp)
                        qq[f][qs][r_][pp] = St::pair(v, pp);
                }
            }
        };

        // prologue: the 2r planes below the first output plane
#pragma unroll
        for (int k = 0; k < 2 * R; ++k) {
            if (ok) {
                if (!wait_or_abort(&full[bar_i], par, abort_flag)) {
                    ok = false;
                } else {
                    load_newest(q, k);
                    __syncwarp();
                    if (lane == 0)
                        mbar_arrive(&empty[bar_i]);
                    advance();
                }
            }
        }
        const int nout = u.z1 - u.z0;
        for (int c0 = 0; c0 < nout && ok; c0 += QN) {
#pragma unroll
            for (int k = 0; k < QN; ++k) {
                const int c = c0 + k;
                if (c < nout && ok) {
                    const int qn = (k + 2 * R) % QN;  // newest plane's queue slot
                    const int qc = (k + R) % QN;      // centre plane's queue slot
                    if (!wait_or_abort(&full[bar_i], par, abort_flag)) {
                        ok = false;
                        break;
                    }
                    load_newest(q, qn);
                    const int slot_c = slot_n >= R ? slot_n - R : slot_n - R + S;
                    // L(u_f) of every field, in the single-step kernel's order
                    float2 sv[NF][PY][PP];
#pragma unroll
                    for (int f = 0; f < NF; ++f) {
                        const unsigned char *cb = slots + (slot_c * NF + f) * slot_bytes + own_off;
                        uint4 ylo[R], yhi[R], xl[PY], xr[PY];
#pragma unroll
                        for (int m = 1; m <= R; ++m) {
                            ylo[m - 1] = lds128(cb - m * ROW_BYTES);
                            yhi[m - 1] = lds128(cb + (PY - 1 + m) * ROW_BYTES);
                        }
#pragma unroll
                        for (int r_ = 0; r_ < PY; ++r_) {
                            xl[r_] = load_left<GBST_F32, R>(cb + r_ * ROW_BYTES - 16);
                            xr[r_] = load_right<GBST_F32, R>(cb + r_ * ROW_BYTES + 16);
                        }
                        auto xel = [&](int r_, int e) -> float {
                            if (e < 0)
                                return St::get(xl[r_], PX + e);
                            if (e >= PX)
                                return St::get(xr[r_], e - PX);
                            return (e & 1) ? q[f][qc][r_][e >> 1].y : q[f][qc][r_][e >> 1].x;
                        };
                        auto yrow = [&](int rr, int pp) -> float2 {
                            if (rr < 0)
                                return St::pair(ylo[-rr - 1], pp);
                            if (rr >= PY)
                                return St::pair(yhi[rr - PY], pp);
                            return q[f][qc][rr][pp];
                        };
#pragma unroll
                        for (int r_ = 0; r_ < PY; ++r_)
#pragma unroll
                            for (int pp = 0; pp < PP; ++pp)
                                sv[f][r_][pp] = __fmul2_rn(wc2, q[f][qc][r_][pp]);
#pragma unroll
                        for (int m = 1; m <= R; ++m) {
#pragma unroll
                            for (int r_ = 0; r_ < PY; ++r_) {
#pragma unroll
                                for (int pp = 0; pp < PP; ++pp) {
                                    const int e = 2 * pp;
                                    const float2 xm = make_float2(xel(r_, e - m), xel(r_, e + 1 - m));
                                    const float2 xp = make_float2(xel(r_, e + m), xel(r_, e + 1 + m));
                                    float2 t = __fadd2_rn(__fadd2_rn(xm, xp),
                                                          __fadd2_rn(yrow(r_ - m, pp), yrow(r_ + m, pp)));
                                    t = __fadd2_rn(t, __fadd2_rn(q[f][(qc - m + 2 * QN) % QN][r_][pp],
                                                                 q[f][(qc + m) % QN][r_][pp]));
                                    sv[f][r_][pp] = __ffma2_rn(w2[m], t, sv[f][r_][pp]);
                                }
                            }
                        }
                    }
                    // all shared-memory reads of this iteration are done: release the planes
                    __syncwarp();
                    if (lane == 0)
                        mbar_arrive(&empty[bar_i]);
                    advance();
#pragma unroll
                    for (int kf = 0; kf < NF; ++kf) {
                        float o[PY][PX];
#pragma unroll
                        for (int r_ = 0; r_ < PY; ++r_)
#pragma unroll
                            for (int pp = 0; pp < PP; ++pp) {
                                float2 ov = q[kf][qc][r_][pp];
#pragma unroll
                                for (int j = 0; j < NF; ++j)
                                    ov = __ffma2_rn(A2[kf][j], sv[j][r_][pp], ov);
                                o[r_][2 * pp] = ov.x;
                                o[r_][2 * pp + 1] = ov.y;
                            }
                        unsigned char *op = outb[kf] + ooff;
#pragma unroll
                        for (int r_ = 0; r_ < PY; ++r_) {
                            if (row_ok[r_]) {
                                if (xfull) {
                                    *reinterpret_cast<uint4 *>(op + r_ * row_stride) = St::pack(o[r_]);
                                } else {
#pragma unroll
                                    for (int i = 0; i < PX; ++i)
                                        if (x0 + i < nx)
                                            St::store1(op + r_ * row_stride + i * ES, o[r_][i]);
                                }
                            }
                        }
                    }
                    ooff += plane_bytes;
                }
            }
        }
    }
    if (!ok)  // a wait gave up (the producer may have left already): report it here
        atomicCAS(a.err, 0, static_cast<int>(kDevTimeoutTma));
}

}  // namespace

template <int R, int NF, int NC, int PY, int D, int MINB, int TXT>
constexpr Entry sys_entry()
{
    StreamVariant v{R, GBST_HEAT, GBST_F32, true, NC * 32, PY, D, MINB, TXT, 1, false};
    v.nf = NF;
    return Entry{v, &k_system<R, NF, NC, PY, D, MINB, TXT>};
}

}  // namespace sweep
}  // namespace gbst
