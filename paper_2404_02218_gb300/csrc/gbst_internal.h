// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "gbstencil.h"

namespace gbst {

constexpr int kMaxRadius = 4;

// Device-side error codes written to the per-handle error word.
enum DevErr : int {
    kDevOk = 0,
    kDevTimeoutTma = 1,     // an mbarrier wait for a TMA plane expired
    kDevTimeoutBarrier = 2, // a grid-wide barrier wait expired
    kDevBadUnit = 3,        // a work unit outside its grid (host bug guard)
};

// Wall-clock limit of every device-side spin wait (nanoseconds, %globaltimer).
constexpr unsigned long long kWaitLimitNs = 2000000000ull;
// Offset (in unsigned ints) of the dynamic-assignment counters in a handle's
// 256-byte grid-barrier buffer.
constexpr int kDynCounterOffset = 16;

// x ghost width in bytes (each side) of the stored fields of wide grids:
// interior rows start on a 128-byte boundary (the row pitch is a multiple of
// 128 bytes too).  Narrow grids keep one 16-byte chunk.
constexpr int kGhostBytesX = 128;

// Padded storage of one field of one (sub)domain.
//   element (i, j, k) of the interior lives at  origin + (k*rows + j)*pitch + i
//   x ghosts: G = kGhostBytesX or 16 bytes, / element size (>= r), each side,
//   y ghosts: r rows, z ghosts: rz = r (3D) or 0 (2D) planes.
//   pitch = round_up(nx + 2G, 128 bytes / element size) elements.
struct Layout {
    int64_t nx = 0, ny = 0, nz = 0;
    int r = 0, rz = 0, G = 0, es = 4;
    int64_t pitch = 0, rows = 0, planes = 0;
    int64_t origin = 0;  // elements
    int64_t elems = 0;   // total allocated elements
    size_t bytes = 0;    // total bytes, rounded up to 256
};

// G: x ghost width in elements.
Layout make_layout(int ndim, int64_t nx, int64_t ny, int64_t nz, int r, int elem_size, int G);

// One (sub)domain as the sweep kernels see it.  Lives in device global memory;
// the tensor maps must be 64-byte aligned.
struct alignas(128) GridDev {
    CUtensorMap tmap[2];   // TMA descriptors of u buffers 0 and 1 (box = tile + halo)
    CUtensorMap tmap_c[2]; // wave: u buffers 0 and 1, interior boxes (tile only)
    CUtensorMap tmap_k;    // wave: kappa, interior boxes
    void *buf[2];          // u buffers (padded, storage type)
    float *kappa;          // wave: kappa (padded FP32 layout `klay`), else null
    int64_t nx, ny, nz;    // interior
    int64_t pitch, rows;   // u layout (elements)
    int64_t origin;        // u layout interior origin (elements)
    int64_t kpitch, krows, korigin;  // kappa layout
    int tiles_x, tiles_y;  // tile grid of this (sub)domain
    int txt;               // threads along x per tile (tile width = txt * PX)
    int box_bytes;         // bytes of one TMA box (tile + halo)
    int src_x, src_y, src_z, has_src;  // source position (interior coordinates)
    float heat_a;          // heat: alpha dt / h^2 of this grid
    int ghost;             // ghost rows / planes of the u layout (r, or 2r for two steps across exchanges)
    int face_int;          // faces shared with another subdomain: bit 2a low, bit 2a + 1 high side of axis a
    CUtensorMap tmap_tb[2];  // two-step kernel: u buffers with all ghost rows and planes (box = tile + 2r halo)
};

// A unit of sweep work: one tile of one grid over planes [z0, z1).
struct Unit {
    int grid, tile, z0, z1;
};

// Per-launch arguments of the sweep kernels.
struct SweepArgs {
    const GridDev *grids;
    const Unit *units;
    int nunits;
    int parity;            // u^n lives in buf[parity]; output goes to buf[1-parity]
    int ndim;
    float wc;              // ndim * w_0 (weights scaled to integers where they are)
    float w[kMaxRadius + 1];  // w_1..w_r at w[1..r]
    float lscale;          // wave: factor on the weighted sum before kappa (1 / the weights' scale)
    const float *srcval;   // wave: per-grid source values, [step][grid] (already scaled), or null
    int *err;              // device error word
    int nsteps;            // steps in this launch (> 1: persistent launch with grid barriers)
    int ngrids;            // grids (row length of srcval)
    unsigned int *barrier; // grid-barrier counter (zeroed before a persistent launch)
    unsigned int barrier_extra;  // test hook: extra arrivals a barrier waits for (0 in normal use)
    int tb_single;         // temporally blocked kernel: 1 = perform one step only
    float coupling[16];    // fused multi-field system: A[k][j] at k * nfields + j
    // Dynamic work assignment of a streaming launch: [0] units drawn beyond the
    // first gridDim, [1] CTAs done (the last CTA of a launch or step zeroes both);
    // null: unit ui goes to CTA ui mod gridDim.
    unsigned int *dyn;
};

// Host-side entry points of the kernel translation units.
struct StreamVariant {
    int R;          // radius
    int eq;         // GBST_HEAT / GBST_WAVE
    int storage;    // GBST_F32 / GBST_BF16
    bool has_z;     // 3D
    int nthreads;   // consumer threads per CTA (one more warp issues the TMA loads)
    int py;         // output rows per thread
    int depth;      // TMA prefetch depth (planes in flight beyond the current one)
    int minb;       // minimum resident CTAs per SM requested from the compiler (register bound)
    int txt;        // threads along x of a tile (tile width = txt * 16 bytes of storage)
    int tb = 1;     // time steps per launch: 1, or 2 (temporally blocked heat kernel)
    bool ys = false; // 2D grid streamed along y (one-row tiles)
    int nf = 1;      // fields of a fused multi-field system sweep (1: a single field)
    int opt = 0;     // streaming-kernel options (kOpt* bits)
};

// Streaming-kernel options.  kOptScalarOddX: the x-neighbour sums of odd
// offsets m (operands that straddle the thread's packed FP32x2 point pairs) as
// two scalar additions each instead of one packed addition of re-paired
// registers (the same results bit for bit).
constexpr int kOptScalarOddX = 2;
// kOptMixedY (BF16 storage): the sum of the two y-neighbour pairs of offset m
// widens the halves of one 32-bit word and adds the other word's halves by
// mixed-precision additions (BF16 + FP32 -> FP32), one widening fewer per pair
// and the same rounded sums bit for bit.
constexpr int kOptMixedY = 4;
// kOptMixedU (BF16 wave): 2u - u^{n-1} as the negated mixed-precision difference
// u^{n-1} - 2u, folded into the final fused multiply-add (the same bits: rounding
// to nearest is symmetric).
constexpr int kOptMixedU = 8;
// Threads of one CTA of a streaming variant (consumers and the producer warp).
inline int block_threads(const StreamVariant &v) { return v.nthreads + 32; }

// Tile of a variant: width in points, height in rows (a temporally blocked
// variant's nthreads counts its main and edge warps; the tile is the grown
// step-1 region of the main warps less r rows on each side).
inline int tile_w(const StreamVariant &v, int px) { return v.txt * px; }
inline int tile_h(const StreamVariant &v)
{
    if (v.ys)
        return 1;
    return v.tb == 2 ? (v.nthreads / 32 - 1) * v.py - 2 * v.R : (v.nthreads / v.txt) * v.py;
}
// Radius along the streaming axis (planes kept below the centre in the ring).
inline int stream_rz(const StreamVariant &v) { return (v.has_z || v.ys) ? v.R : 0; }

// Number of element columns a thread owns (16 bytes of storage).
inline int px_of(int storage) { return storage == GBST_BF16 ? 8 : 4; }

// Shared-memory bytes of the streaming kernel for the given variant and max box size.
size_t stream_smem_bytes(const StreamVariant &v, int max_box_bytes);
// Plane-slot bytes of a launch with `smem` bytes of shared memory.
int stream_slot_bytes(const StreamVariant &v, size_t smem);
// Launch the streaming (TMA, 2.5D) sweep.  Returns cudaSuccess or the launch error.
cudaError_t launch_stream_sweep(const StreamVariant &v, const SweepArgs &a, int ctas, size_t smem,
                                cudaStream_t s, bool cooperative = false);
// Max resident CTAs per SM of the variant at the given shared memory size (0 = unsupported).
int stream_occupancy(const StreamVariant &v, size_t smem);
bool stream_variant_exists(const StreamVariant &v);
int stream_variant_count();
bool stream_variant_get(int i, StreamVariant *v);

// Simple kernel: one thread per output point, plain global loads.
cudaError_t launch_simple_sweep(int R, int eq, int storage, const SweepArgs &a, int ngrids,
                                int64_t max_points, cudaStream_t s);

// Halo copies (dmp.swap faces, periodic wrap): a list of boxes copied element-wise.
struct CopyBox {
    int64_t src_off, dst_off;  // bytes from the subdomain base pointers
    int src_grid, dst_grid;
    int64_t ex, ey, ez;        // extents (elements)
    int blk0, nblk;            // this box's blocks [blk0, blk0 + nblk) of the copy launch
};
// Block counts of one copy launch: sets blk0 / nblk of every box, returns the total.
int halo_copy_blocks(CopyBox *boxes, int nboxes);
cudaError_t launch_halo_copies(const GridDev *grids, const CopyBox *boxes, int nboxes, int parity,
                               int elem_size, int total_blocks, cudaStream_t s);

// Field transfer kernels between dense (x fastest) and padded storage.
// dense dtype: GBST_F32 / GBST_F64 / GBST_BF16.  Region: the subdomain interior
// located at global offset (gx, gy, gz) of a dense global field (gnx, gny, gnz).
struct XferArgs {
    void *padded; int storage; int64_t pitch, rows, origin;  // padded field
    int64_t nx, ny, nz;                                       // subdomain interior
    int64_t gx, gy, gz, gnx, gny;                             // placement in the dense field
    void *dense; int dense_dtype;
    double scale_sq;   // VEL -> kappa: kappa = c^2 * scale_sq (0 = plain copy)
};
cudaError_t launch_scatter(const XferArgs &x, cudaStream_t s);
cudaError_t launch_gather(const XferArgs &x, cudaStream_t s);
// padded[o] += dense (FP32 dense, storage F32 or BF16)
cudaError_t launch_scatter_add(const XferArgs &x, cudaStream_t s);
// dense[ (k/st*ceil(ny/st) + j/st) * ceil(nx/st) + i/st ] = padded(i, j, k) for i, j, k multiples of st
cudaError_t launch_gather_strided(const XferArgs &x, int stride, cudaStream_t s);
// c_norm = sqrt(kappa) * h / (dt * c_ref), dense FP32 from the padded kappa field
cudaError_t launch_kappa_to_cnorm(const XferArgs &x, double factor, cudaStream_t s);

// FP64 reductions.  kinds as GBST_RED_*.  Partials: one double per block.
struct ReduceGrid {
    const void *u; const void *v; const float *kappa;  // v = u^{n-1} (energy)
    int64_t pitch, rows, origin, kpitch, krows, korigin;
    int64_t nx, ny, nz;
};
int reduce_blocks_for(int64_t points);
cudaError_t launch_reduce_partials(int kind, int storage, int ndim, int R, const double *w,
                                   const ReduceGrid *grids_dev, int ngrids, int64_t max_points,
                                   double *partials, int nblocks, cudaStream_t s);
cudaError_t launch_reduce_final(int kind, const double *partials, int n, double *out,
                                cudaStream_t s);

// Stream a closure was created on.
cudaStream_t closure_stream(gbst_closure c);

// Record the message returned by stencil_last_error() for the calling thread.
gbst_status record_error(gbst_status st, const char *msg);
// Dense-array stencils of the closure (closure_train.cu).
gbst_status dense_star(int r, const double *w, int64_t nx, int64_t ny, int64_t nz, const float *in, const float *pre,
                       const float *post, double alpha, bool accumulate, float *out, cudaStream_t s);
struct ClosureFeatBufs {
    float *cn2 = nullptr, *g[3] = {nullptr, nullptr, nullptr}, *lu = nullptr, *t5 = nullptr, *t6 = nullptr,
          *e7 = nullptr, *tmp = nullptr;  // dense, one value per point each
};
gbst_status closure_features_forward(const float *up, const float *un, const float *cn, int64_t nx, int64_t ny,
                                     int64_t nz, int r, const double *w, const double *scales,
                                     const ClosureFeatBufs &b, __nv_bfloat16 *x, bool aux, int xch, cudaStream_t s);
gbst_status closure_features_adjoint(const __nv_bfloat16 *dx, int64_t nx, int64_t ny, int64_t nz, int r,
                                     const double *w, const double *scales, const ClosureFeatBufs &b, float *g_up,
                                     float *g_un, cudaStream_t s);
bool closure_has_features(gbst_closure c);
gbst_status rollout_sums(const float *u, const float *ref, int64_t n, double *sums, cudaStream_t s);
gbst_status rollout_grad(float *u, const float *ref, int64_t n, const double *sums, double scale, cudaStream_t s);
gbst_status dense_axpy(float *y, const float *x, float a, int64_t n, cudaStream_t s);
gbst_status closure_features_values(const float *up, const float *un, int64_t nx, int64_t ny, int64_t nz,
                                    const ClosureFeatBufs &b, float *out, cudaStream_t s);

// Tensor-map encoding through the driver entry point.
// Tiled tensor map of a 4D BF16 tensor (dims innermost first; strides in bytes of dims 1..3);
// swizzle32: boxes land in the 32-byte swizzled shared-memory layout (inner box extent 32 bytes).
bool encode_tmap_bf16_4d(CUtensorMap *m, const void *base, const uint64_t dims[4], const uint64_t strides[3],
                         const uint32_t box[4], std::string *err, bool swizzle32 = false);
// Tiled tensor map of a padded field: x from `lead` elements before the interior,
// `reach` ghost rows / planes on each side (-1: all of the layout's).
bool encode_tmap(CUtensorMap *m, void *base, const Layout &L, int storage, int box_w, int box_h, int lead,
                 std::string *err, int reach);

}  // namespace gbst
