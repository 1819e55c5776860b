// C-ABI implementation: handles, field layout, decomposition (dmp.swap
// exchanges), execution planning, TMA descriptors, CUDA-graph capture of the
// step loop, field transfers and reductions.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include <cudaTypedefs.h>

#include "gbst_internal.h"

namespace gbst {

// ---------------------------------------------------------------- errors ---
static thread_local std::string t_err;

static bool log_enabled()
{
    static const bool on = [] {
        const char *e = getenv("GBST_LOG");
        return e && e[0] == '1';
    }();
    return on;
}

static gbst_status fail(gbst_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    t_err = buf;
    if (log_enabled())
        fprintf(stderr, "[gbstencil] %s\n", buf);
    return st;
}

gbst_status record_error(gbst_status st, const char *msg) { return fail(st, "%s", msg); }

#define GBST_CUDA(call)                                                                             \
    do {                                                                                            \
        cudaError_t e_ = (call);                                                                    \
        if (e_ != cudaSuccess)                                                                      \
            return fail(GBST_ECUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, \
                        __LINE__);                                                                  \
    } while (0)

// ---------------------------------------------------------------- layout ---
Layout make_layout(int ndim, int64_t nx, int64_t ny, int64_t nz, int r, int es, int G)
{
    Layout L;
    L.nx = nx;
    L.ny = ny;
    L.nz = ndim == 3 ? nz : 1;
    L.r = r;
    L.rz = ndim == 3 ? r : 0;
    L.G = G;
    L.es = es;
    const int64_t align = 128 / es;
    L.pitch = (nx + 2 * G + align - 1) / align * align;
    L.rows = ny + 2 * r;
    L.planes = L.nz + 2 * L.rz;
    L.origin = (L.rz * L.rows + r) * L.pitch + G;
    L.elems = L.pitch * L.rows * L.planes;
    L.bytes = (static_cast<size_t>(L.elems) * es + 255) / 256 * 256;
    return L;
}

static PFN_cuTensorMapEncodeTiled_v12000 tmap_encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

bool encode_tmap_bf16_4d(CUtensorMap *m, const void *base, const uint64_t dims[4], const uint64_t strides[3],
                         const uint32_t box[4], std::string *err, bool swizzle32)
{
    auto fn = tmap_encoder();
    if (!fn) {
        *err = "cuTensorMapEncodeTiled is not available from the driver";
        return false;
    }
    cuuint64_t d[4], st[3];
    cuuint32_t b[4], es[4] = {1, 1, 1, 1};
    for (int i = 0; i < 4; ++i) {
        d[i] = dims[i];
        b[i] = box[i];
    }
    for (int i = 0; i < 3; ++i)
        st[i] = strides[i];
    CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void *>(base), d, st, b, es,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle32 ? CU_TENSOR_MAP_SWIZZLE_32B : CU_TENSOR_MAP_SWIZZLE_NONE,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        *err = "cuTensorMapEncodeTiled failed (" + std::to_string(static_cast<int>(r)) + ") for a 4D BF16 tensor";
        return false;
    }
    return true;
}

// Tensor map of a padded field.  The kernels address x from `lead` elements
// before the interior (one 16-byte chunk of the storage type), so the map
// starts L.G - lead elements into each row (L.G >= lead) and covers the
// interior and `lead` ghosts on each side: boxes that reach further read
// zeros without touching the row padding.
bool encode_tmap(CUtensorMap *m, void *base, const Layout &L, int storage, int box_w, int box_h, int lead,
                 std::string *err, int reach)
{
    auto fn = tmap_encoder();
    if (!fn) {
        *err = "cuTensorMapEncodeTiled is not available from the driver";
        return false;
    }
    // ghost rows / planes the map covers (coordinate 0 = the first of them)
    const int ry = reach < 0 ? L.r : std::min(reach, L.r), rz = reach < 0 ? L.rz : std::min(reach, L.rz);
    const int64_t shift = L.G - lead + ((L.rz - rz) * L.rows + (L.r - ry)) * L.pitch;
    base = static_cast<unsigned char *>(base) + shift * L.es;
    const cuuint64_t dims[3] = {static_cast<cuuint64_t>(L.nx + 2 * lead), static_cast<cuuint64_t>(L.ny + 2 * ry),
                                static_cast<cuuint64_t>(L.nz + 2 * rz)};
    const cuuint64_t strides[2] = {static_cast<cuuint64_t>(L.pitch) * L.es,
                                   static_cast<cuuint64_t>(L.pitch) * L.rows * L.es};
    const cuuint32_t box[3] = {static_cast<cuuint32_t>(box_w), static_cast<cuuint32_t>(box_h), 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUtensorMapDataType dt =
        storage == GBST_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    // L2 promotion: 64 bytes for rows of at least 2 KB (with 128 or 256 bytes the order-8
    // sweep at 512^3 read 1.18 x the field from DRAM, with 64 bytes 1.11 x, in the same
    // time; the wide-row sweeps are equal or slightly faster), 256 bytes for shorter rows
    // (the 64-grid batch of 96-256-point rows ran 2 % slower with 64)
    const CUtensorMapL2promotion promo =
        L.nx * L.es >= 2048 ? CU_TENSOR_MAP_L2_PROMOTION_L2_64B : CU_TENSOR_MAP_L2_PROMOTION_L2_256B;
    CUresult r = fn(m, dt, 3, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_NONE, promo, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        char b[160];
        snprintf(b, sizeof b, "cuTensorMapEncodeTiled failed (%d) for box %dx%d, dims %lld x %lld x %lld",
                 static_cast<int>(r), box_w, box_h, static_cast<long long>(L.pitch),
                 static_cast<long long>(L.rows), static_cast<long long>(L.planes));
        *err = b;
        return false;
    }
    return true;
}

// Central second-derivative weights of accuracy 2r, closed form:
//   w_m = 2 (-1)^{m+1} (r!)^2 / (m^2 (r-m)! (r+m)!),  w_0 = -2 sum_{m>=1} w_m.
static void central_weights(int r, double *w)
{
    auto fact = [](int n) {
        double f = 1.0;
        for (int i = 2; i <= n; ++i)
            f *= i;
        return f;
    };
    double s = 0.0;
    for (int m = 1; m <= r; ++m) {
        const double v = 2.0 * ((m + 1) % 2 == 0 ? 1.0 : -1.0) * fact(r) * fact(r) /
                         (static_cast<double>(m) * m * fact(r - m) * fact(r + m));
        w[m] = v;
        s += v;
    }
    w[0] = -2.0 * s;
}

// max over theta of |w_0 + 2 sum_m w_m cos(m theta)|, sampled densely (the
// standard weights peak at theta = pi; caller weights may peak elsewhere).
static double symbol_max(int r, const double *w)
{
    double best = 0.0;
    const int n = 4096;
    for (int i = 0; i <= n; ++i) {
        const double th = M_PI * i / n;
        double v = w[0];
        for (int m = 1; m <= r; ++m)
            v += 2.0 * w[m] * cos(m * th);
        best = std::max(best, std::fabs(v));
    }
    return best;
}

// ---------------------------------------------------------------- memory ---
struct Allocator {
    gbst_allocator a{};
    bool custom = false;
    cudaStream_t s = nullptr;
    void *alloc(size_t bytes)
    {
        if (bytes == 0)
            bytes = 256;
        if (custom)
            return a.alloc(bytes, s, a.ctx);
        void *p = nullptr;
        if (cudaMalloc(&p, bytes) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        return p;
    }
    void release(void *p, size_t bytes)
    {
        if (!p)
            return;
        if (custom)
            a.release(p, bytes, s, a.ctx);
        else
            cudaFree(p);
    }
};

struct DevMem {
    void *p = nullptr;
    size_t bytes = 0;
};

}  // namespace gbst

using namespace gbst;

struct Sub {
    Layout lu, lk;
    int64_t g0[3];      // offset of the interior in the caller's dense arrays (x, y, z)
    int64_t dense[3];   // dims of those dense arrays: the whole grid, or the batch member itself
    int c[3];           // coordinates in the decomposition grid
    int member = 0;     // batch member (0 for a single, possibly decomposed, grid)
    double dt = 0.0, h = 1.0, alpha = 0.0;
    // Ricker point source of the wave equation
    bool src_on = false;
    int64_t src_local[3] = {0, 0, 0};
    double f0 = 0.0, t0 = 0.0, amp = 0.0, kappa_src = 0.0;
    bool unstable = false;  // kappa above the stability limit
};

// Rows of at least this many bytes get kGhostBytesX-wide x ghosts; narrower rows
// keep one 16-byte chunk (measured below, where the layouts are made).
constexpr int64_t kWideRowBytes = 2048;

// Default unit assignment of streaming launches: dynamic (measured equal or
// faster for every streaming variant; fewer DRAM re-reads of halo planes).
constexpr bool kDynDefault = true;
// Default of the halo-exchange overlap (decomposition mode, periodic wrap): off.
// On one device the face copies are a small part of a step, and splitting the
// sweep costs more than they take (1024^3 order 4 on 2x2x2 subdomains: 58 % of
// the units read an exchanged face; 672 GPoints/s overlapped, 711 plain).
constexpr bool kOverlapDefault = false;

struct Plan {
    StreamVariant var{};
    int variant = -1;
    int req_txt = 0, req_zchunks = 0, req_ctas = 0;
    bool stream = false;
    int txt = 16;
    int zchunks = 1;
    int ctas = 0;
    size_t smem = 0;
    int occupancy = 0;
    int nunits = 0;
    int max_box_bytes = 0;
    bool dyn = false;  // launches draw their work units from a global counter
    // halo exchanges overlapped with the sweep: units [0, nint) read no exchanged
    // ghost cell and sweep while the copies run; units [nint, nunits) sweep after them
    bool overlap = false;
    int nint = 0;
};

struct gbst_grid_s {
    gbst_desc d{};
    int ndim = 3, R = 1, es = 4;
    double w[kMaxRadius + 1] = {0};
    // the weights as integers over a common denominator wscale where they are (the central
    // weights: 1, 12 and 5040 for orders 2, 4 and 8), else wint = w and wscale = 1
    double wint[kMaxRadius + 1] = {0};
    double wscale = 1.0;
    double S = 0.0;
    int decomp[3] = {1, 1, 1};
    bool batch = false;
    int members = 1;
    int nf = 1;               // fused multi-field system: the members are its fields
    float coupling[16] = {0}; // system coupling matrix A[k][j] (k * nf + j)
    cudaStream_t stream = nullptr;
    Allocator mem;
    std::vector<DevMem> owned;
    std::vector<Sub> subs;
    std::vector<GridDev> hgrids;
    GridDev *dgrids = nullptr;
    Unit *dunits = nullptr;
    size_t units_cap = 0;
    CopyBox *dboxes = nullptr;
    int nboxes = 0;
    int64_t max_box_elems = 0;
    int copy_blocks = 0;  // blocks of one halo copy launch
    // Two time steps across exchanges (decomposed heat grids): ghost regions 2r deep and
    // a second copy list, run before every two-step launch in three phases (x, y, then z
    // faces, each spanning the ghost cells the earlier phases filled).
    bool deep = false;
    CopyBox *ddeep = nullptr;
    int deep_n[3] = {0, 0, 0};       // boxes of each phase (consecutive in ddeep)
    int deep_blocks[3] = {0, 0, 0};  // blocks of each phase's launch
    int64_t max_points = 0;
    Plan plan;
    int parity = 0;
    int64_t step = 0;
    int *derr = nullptr;
    unsigned int *dbarrier = nullptr;
    unsigned int barrier_extra = 0;
    int dyn_pref = -1;  // unit assignment of streaming launches: -1 default, 0 static, 1 dynamic
    int overlap_pref = -1;  // halo exchange overlapped with the sweep: -1 default, 0 off, 1 on
    cudaStream_t side = nullptr;  // stream of the overlapped halo copies
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    bool persistent = false;
    double *dpartials = nullptr;
    int red_blocks_per_grid = 0;
    double *dred_out = nullptr;
    ReduceGrid *dred_grids = nullptr;
    float *dsrc = nullptr;
    float *hsrc = nullptr;
    int64_t src_cap = 0;  // steps
    cudaEvent_t src_ev = nullptr;
    gbst_status sticky = GBST_OK;
    std::map<std::pair<int64_t, int>, cudaGraphExec_t> graphs;
    bool profile = false;
    std::vector<cudaEvent_t> prof_ev;
    int64_t prof_launches = 0;
    // learned closure applied after every sweep (single 3D wave grid)
    gbst_closure closure = nullptr;
    float *cl_up = nullptr, *cl_un = nullptr, *cl_cn = nullptr, *cl_corr = nullptr;
    // training the attached closure through rollouts (stencil_closure_rollout_grad)
    std::vector<float *> roll_up, roll_un, roll_u;  // per step: u+, u^n, u^{n+1} (then its loss gradient)
    float *roll_a[3] = {nullptr, nullptr, nullptr};  // cotangents of three consecutive levels
    float *roll_A = nullptr, *roll_gun = nullptr, *roll_kap = nullptr;
    double *roll_sums = nullptr;  // 2 per step
    int roll_cap = 0;
};

namespace {

int num_sms()
{
    static int n = [] {
        int dev = 0, v = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        return v > 0 ? v : 1;
    }();
    return n;
}

void *dalloc(gbst_handle h, size_t bytes)
{
    void *p = h->mem.alloc(bytes);
    if (p)
        h->owned.push_back(DevMem{p, bytes});
    return p;
}

void dfree(gbst_handle h, void *p)
{
    for (size_t i = 0; i < h->owned.size(); ++i)
        if (h->owned[i].p == p) {
            h->mem.release(p, h->owned[i].bytes);
            h->owned.erase(h->owned.begin() + i);
            return;
        }
}

gbst_status check_handle(gbst_handle h)
{
    if (!h)
        return fail(GBST_EINVAL, "null handle");
    if (h->sticky == GBST_ECUDA || h->sticky == GBST_ETIMEOUT)
        return fail(h->sticky, "handle is poisoned by an earlier device error");
    return GBST_OK;
}

// Read the device error word; converts a device-side failure into a sticky status.
gbst_status poll_device_error(gbst_handle h)
{
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
        h->sticky = GBST_ECUDA;
        return fail(GBST_ECUDA, "device error: %s", cudaGetErrorString(e));
    }
    int code = 0;
    e = cudaMemcpy(&code, h->derr, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
        h->sticky = GBST_ECUDA;
        return fail(GBST_ECUDA, "reading the device error word: %s", cudaGetErrorString(e));
    }
    if (code != kDevOk) {
        h->sticky = GBST_ETIMEOUT;
        return fail(GBST_ETIMEOUT, "a bounded device-side wait expired (code %d)", code);
    }
    return GBST_OK;
}

void destroy_graphs(gbst_handle h)
{
    for (auto &kv : h->graphs)
        cudaGraphExecDestroy(kv.second);
    h->graphs.clear();
}

// ---- plan: tiles, TMA boxes, work units ----------------------------------
// Index of the first streaming variant matching the handle (the default), or -1.
// Two-step (temporally blocked) sweeps need a heat grid in FP32, 3D, with zero
// ghosts and no halo exchange between steps.
bool tb_allowed(gbst_handle h)
{
    return h->nf == 1 && h->d.temporal_block != 1 && h->d.eq == GBST_HEAT && h->d.storage == GBST_F32 && h->ndim == 3 &&
           h->d.bc == GBST_BC_ZERO && (h->nboxes == 0 || h->deep) && h->d.kernel != GBST_KERNEL_SIMPLE;
}

bool variant_matches(gbst_handle h, const StreamVariant &v)
{
    if (v.R != h->R || v.eq != h->d.eq || v.storage != h->d.storage || v.has_z != (h->ndim == 3) || v.nf != h->nf)
        return false;
    return v.tb == 1 || tb_allowed(h);
}

int default_variant(gbst_handle h)
{
    StreamVariant v;
    const int want_tb = h->d.temporal_block == 2 && tb_allowed(h) ? 2 : 1;
    for (int i = 0; stream_variant_get(i, &v); ++i)
        if (variant_matches(h, v) && v.tb == want_tb)
            return i;
    return -1;
}

gbst_status build_plan(gbst_handle h, int variant, int txt, int zchunks_req, int ctas_req)
{
    const int st = h->d.storage;
    const int px = px_of(st);
    const int G = px;
    Plan p;
    if (variant < 0)
        variant = default_variant(h);
    p.stream = h->d.kernel != GBST_KERNEL_SIMPLE && variant >= 0;
    if ((h->d.kernel == GBST_KERNEL_STREAM || h->nf > 1) && !p.stream)
        return fail(GBST_ENOTSUP, "no streaming kernel for radius %d%s", h->R,
                    h->nf > 1 ? " and this number of fields" : "");
    if (p.stream) {
        if (!stream_variant_get(variant, &p.var))
            return fail(GBST_EINVAL, "unknown kernel variant %d", variant);
        if (!variant_matches(h, p.var))
            return fail(GBST_EINVAL, "kernel variant %d does not match this grid", variant);
        p.variant = variant;
    } else {
        p.var = StreamVariant{h->R, h->d.eq, st, h->ndim == 3, 128, 1, 1, 1, 8};
    }
    const int nt = p.var.nthreads;
    // tile: txt threads along x (fixed by the variant), nt / txt along y
    if (!p.stream)
        p.var.txt = 8;
    if (p.stream && txt != 0 && txt != p.var.txt)
        return fail(GBST_EINVAL, "txt %d does not match kernel variant %d (tile of %d threads in x)", txt, variant,
                    p.var.txt);
    p.txt = p.var.txt;
    (void)nt;
    const int TX = tile_w(p.var, px), TY = tile_h(p.var);
    // two-step variants read the tile plus 2 chunks in x and 2r rows in y per side;
    // y-streaming (2D) variants read one row per plane
    const bool ys = p.stream && p.var.ys;
    const int box_w = TX + 2 * G * p.var.tb, box_h = ys ? 1 : TY + 2 * h->R * p.var.tb;
    if (box_w > 256 || box_h > 256)
        return fail(GBST_EINVAL, "tile %dx%d too large for a TMA box", TX, TY);
    p.max_box_bytes = box_w * box_h * h->es;

    int64_t T = 0;
    for (size_t i = 0; i < h->subs.size(); ++i) {
        GridDev &g = h->hgrids[i];
        const Sub &s = h->subs[i];
        g.txt = p.txt;
        g.tiles_x = static_cast<int>((s.lu.nx + TX - 1) / TX);
        g.tiles_y = ys ? 1 : static_cast<int>((s.lu.ny + TY - 1) / TY);
        g.box_bytes = p.max_box_bytes;
        if (h->nf == 1 || i == 0)  // a system sweeps the tiles of field 0 only
            T += static_cast<int64_t>(g.tiles_x) * g.tiles_y;
        if (p.stream) {
            std::string err;
            for (int b = 0; b < 2; ++b)
                if (!encode_tmap(&g.tmap[b], g.buf[b], s.lu, st, box_w, box_h, px, &err, h->R) ||
                    (p.var.tb == 2 && !encode_tmap(&g.tmap_tb[b], g.buf[b], s.lu, st, box_w, box_h, px, &err, -1)))
                    return fail(GBST_ECUDA, "%s", err.c_str());
            if (h->d.eq == GBST_WAVE) {
                for (int b = 0; b < 2; ++b)
                    if (!encode_tmap(&g.tmap_c[b], g.buf[b], s.lu, st, TX, TY, px, &err, h->R))
                        return fail(GBST_ECUDA, "%s", err.c_str());
                if (!encode_tmap(&g.tmap_k, g.kappa, s.lk, GBST_F32, TX, TY, px, &err, h->R))
                    return fail(GBST_ECUDA, "%s", err.c_str());
            }
        }
    }
    if (p.stream) {
        p.smem = stream_smem_bytes(p.var, p.max_box_bytes);
        p.occupancy = stream_occupancy(p.var, p.smem);
        if (p.occupancy <= 0)
            return fail(GBST_ENOTSUP, "streaming kernel does not fit (smem %zu)", p.smem);
        const int64_t cmax = static_cast<int64_t>(p.occupancy) * num_sms();
        // extent along the streaming axis: z (3D) or y (2D streamed along y)
        const int64_t nz = ys ? h->subs[0].lu.ny : h->subs[0].lu.nz;
        int zc = 1;
        if (h->ndim == 3 || ys) {
            if (zchunks_req > 0) {
                zc = static_cast<int>(std::min<int64_t>(zchunks_req, nz));
            } else {
                // minimise waves * (chunk length + 2r): a balance / halo-overhead trade-off
                double best = 1e300;
                for (int c = 1; c <= 64 && nz / c >= 2 * h->R + 1; ++c) {
                    const int64_t units = T * c;
                    const int64_t waves = (units + cmax - 1) / cmax;
                    const double cost = static_cast<double>(waves) * ((nz + c - 1) / c + 2 * h->R * p.var.tb);
                    if (cost < best * 0.999) {
                        best = cost;
                        zc = c;
                    }
                }
            }
        }
        // dynamic unit assignment
        p.dyn = h->dyn_pref == 1 || (h->dyn_pref < 0 && kDynDefault);
        p.zchunks = zc;
        // Overlap of the halo exchange with the sweep (single-step plans with copies):
        // the units whose TMA boxes reach an exchanged ghost region go last.
        const bool split = h->nboxes > 0 && p.var.tb == 1 && !ys && h->nf == 1 &&
                           (h->overlap_pref == 1 || (h->overlap_pref < 0 && kOverlapDefault));
        auto exchanged = [&](const Sub &s, int a, int dir) {
            if (h->d.bc == GBST_BC_PERIODIC)
                return a < h->ndim;
            const int nb = s.c[a] + dir;
            return nb >= 0 && nb < h->decomp[a];
        };
        std::vector<Unit> units, late;
        for (int c = 0; c < zc; ++c)
            for (size_t i = 0; i < h->subs.size(); ++i) {
                if (h->nf > 1 && i > 0)
                    break;  // a system sweep reads and writes all its fields from the units of field 0
                const GridDev &g = h->hgrids[i];
                const Sub &s = h->subs[i];
                const int64_t n = ys ? s.lu.ny : s.lu.nz;
                const int z0 = static_cast<int>(n * c / zc), z1 = static_cast<int>(n * (c + 1) / zc);
                if (z1 <= z0)
                    continue;
                for (int t = 0; t < g.tiles_x * g.tiles_y; ++t) {
                    const Unit u{static_cast<int>(i), t, z0, z1};
                    bool reach = false;
                    if (split) {
                        // box: x [bx - one chunk, bx + TX + one chunk), y [by - r, by + TY + r),
                        // z [z0 - r, z1 + r)
                        const int64_t bx = static_cast<int64_t>(t % g.tiles_x) * TX;
                        const int64_t by = static_cast<int64_t>(t / g.tiles_x) * TY;
                        reach = (bx == 0 && exchanged(s, 0, -1)) || (bx + TX + G > s.lu.nx && exchanged(s, 0, 1)) ||
                                (h->ndim >= 2 && by == 0 && exchanged(s, 1, -1)) ||
                                (h->ndim >= 2 && by + TY + h->R > s.lu.ny && exchanged(s, 1, 1)) ||
                                (h->ndim == 3 && z0 == 0 && exchanged(s, 2, -1)) ||
                                (h->ndim == 3 && z1 + h->R > s.lu.nz && exchanged(s, 2, 1));
                    }
                    (reach ? late : units).push_back(u);
                }
            }
        p.nint = static_cast<int>(units.size());
        p.overlap = split && p.nint > 0 && !late.empty();
        if (!p.overlap)
            p.nint = 0;
        units.insert(units.end(), late.begin(), late.end());
        p.nunits = static_cast<int>(units.size());
        p.ctas = static_cast<int>(std::min<int64_t>(p.nunits, ctas_req > 0 ? ctas_req : cmax));
        if (units.size() > h->units_cap) {
            if (h->dunits)
                dfree(h, h->dunits);
            h->dunits = static_cast<Unit *>(dalloc(h, units.size() * sizeof(Unit)));
            if (!h->dunits)
                return fail(GBST_ENOMEM, "work-unit list");
            h->units_cap = units.size();
        }
        GBST_CUDA(cudaMemcpyAsync(h->dunits, units.data(), units.size() * sizeof(Unit), cudaMemcpyHostToDevice,
                                  h->stream));
    }
    GBST_CUDA(cudaMemcpyAsync(h->dgrids, h->hgrids.data(), h->hgrids.size() * sizeof(GridDev),
                              cudaMemcpyHostToDevice, h->stream));
    GBST_CUDA(cudaStreamSynchronize(h->stream));
    p.req_txt = txt;
    p.req_zchunks = zchunks_req;
    p.req_ctas = ctas_req;
    h->plan = p;
    destroy_graphs(h);
    return GBST_OK;
}

// ---- autotuner cache --------------------------------------------------------
struct TunedPlan {
    int variant, txt, zchunks, ctas, dyn;
};

std::mutex g_tune_mu;
std::map<std::string, TunedPlan> g_tune_cache;
bool g_tune_loaded = false;

std::string tune_key(gbst_handle h)
{
    // shape class: the first subdomain's sizes plus a hash of every subdomain's sizes
    uint64_t hash = 1469598103934665603ull;
    for (const Sub &s : h->subs)
        for (int64_t v : {s.lu.nx, s.lu.ny, s.lu.nz}) {
            hash ^= static_cast<uint64_t>(v);
            hash *= 1099511628211ull;
        }
    char b[256];
    snprintf(b, sizeof b, "sm%d/r%d/eq%d/st%d/nd%d/%lldx%lldx%lld/sub%zu/%016llx", num_sms(), h->R, h->d.eq,
             h->d.storage, h->ndim, static_cast<long long>(h->subs[0].lu.nx), static_cast<long long>(h->subs[0].lu.ny),
             static_cast<long long>(h->subs[0].lu.nz), h->subs.size(), static_cast<unsigned long long>(hash));
    return b;
}

// Cache file (GBST_TUNE_CACHE): one "key variant txt zchunks ctas dyn" line per entry.
void tune_cache_load()
{
    if (g_tune_loaded)
        return;
    g_tune_loaded = true;
    const char *path = getenv("GBST_TUNE_CACHE");
    if (!path)
        return;
    FILE *f = fopen(path, "r");
    if (!f)
        return;
    char line[512], key[256];
    while (fgets(line, sizeof line, f)) {
        TunedPlan t{0, 0, 0, 0, -1};
        if (sscanf(line, "%255s %d %d %d %d %d", key, &t.variant, &t.txt, &t.zchunks, &t.ctas, &t.dyn) >= 5)
            g_tune_cache[key] = t;
    }
    fclose(f);
}

void tune_cache_store(const std::string &key, const TunedPlan &t)
{
    g_tune_cache[key] = t;
    const char *path = getenv("GBST_TUNE_CACHE");
    if (!path)
        return;
    FILE *f = fopen(path, "a");
    if (!f)
        return;
    fprintf(f, "%s %d %d %d %d %d\n", key.c_str(), t.variant, t.txt, t.zchunks, t.ctas, t.dyn);
    fclose(f);
}

bool tune_cache_find(gbst_handle h, TunedPlan *t)
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    tune_cache_load();
    auto it = g_tune_cache.find(tune_key(h));
    if (it == g_tune_cache.end())
        return false;
    *t = it->second;
    return true;
}

// ---- halo copy list: dmp.swap exchanges (decomposition) or periodic wrap --
struct Exch {
    int64_t at[3], size[3], off[3];
    int to[3];
};

// Exchanges of one subdomain, following Section 4.2: receive into [at, at+size)
// from the neighbour at relative position `to`, send [at+off, at+off+size).
// Coordinates are interior-relative (ghosts at negative / >= n indices).
std::vector<Exch> exchanges(const Sub &s, const int grid[3], int ndim, int R)
{
    std::vector<Exch> out;
    const int64_t n[3] = {s.lu.nx, s.lu.ny, s.lu.nz};
    for (int a = 0; a < ndim; ++a)
        for (int dir = -1; dir <= 1; dir += 2) {
            const int nb = s.c[a] + dir;
            if (nb < 0 || nb >= grid[a])
                continue;
            Exch e{};
            for (int b = 0; b < 3; ++b) {
                if (b == a) {
                    e.at[b] = dir < 0 ? -R : n[b];
                    e.size[b] = R;
                    e.off[b] = dir < 0 ? R : -R;
                    e.to[b] = dir;
                } else {
                    e.at[b] = 0;
                    e.size[b] = b < ndim ? n[b] : 1;
                    e.off[b] = 0;
                    e.to[b] = 0;
                }
            }
            out.push_back(e);
        }
    return out;
}

int64_t byte_off(const Layout &L, int64_t i, int64_t j, int64_t k)
{
    return ((k + L.rz) * L.rows + (j + L.r)) * L.pitch * L.es + (i + L.G) * L.es;
}

// An x face (rows of r elements, each its own DRAM sector at both ends) widened to
// whole 32-byte sectors: receive [-W, 0) from the sender's last W interior columns,
// or [n, n + W) from its first W.  The extra ghost cells lie beyond the radius and
// are never read; writing whole sectors spares the DRAM fills of partly written ones.
// Only where both x ghost regions hold W elements and the sender has W columns.
void widen_x_face(CopyBox &b, const Layout &dst, const Layout &src, int dir, int R)
{
    const int W = 32 / dst.es;
    if (R >= W || dst.G < W || src.G < W || src.nx < W)
        return;
    if (dir < 0) {
        b.dst_off -= static_cast<int64_t>(W - R) * dst.es;
        b.src_off -= static_cast<int64_t>(W - R) * src.es;
    }
    b.ex = W;
}

// Exchange before a two-step launch (deep ghosts, decomposition only): faces 2r deep
// and the edge regions two steps of a star stencil reach (r x r across two axes).
// Three phases, each a launch: x faces; y faces over x from one 16-byte chunk before
// to one after the interior (the neighbour's x ghosts, filled in phase 0, are our
// x-y edges); z faces over those x columns and y from -2r to ny + 2r (the x-z and
// y-z edges).  Every received cell is the value the neighbour holds at the same
// global point, so the two-step kernel sees what it would see undecomposed.
gbst_status build_deep_copies(gbst_handle h)
{
    const int D = 2 * h->R;
    std::vector<CopyBox> ph[3];
    auto index_of = [&](const int c[3]) { return (c[2] * h->decomp[1] + c[1]) * h->decomp[0] + c[0]; };
    for (size_t i = 0; i < h->subs.size(); ++i) {
        const Sub &s = h->subs[i];
        const int64_t n[3] = {s.lu.nx, s.lu.ny, s.lu.nz};
        const int X = 16 / h->es;  // x ghost columns carried by the y and z faces
        for (int a = 0; a < 3; ++a)
            for (int dir = -1; dir <= 1; dir += 2) {
                int nc[3] = {s.c[0], s.c[1], s.c[2]};
                nc[a] += dir;
                if (nc[a] < 0 || nc[a] >= h->decomp[a])
                    continue;
                const int ni = index_of(nc);
                const Sub &ns = h->subs[ni];
                const int64_t nn = a == 0 ? ns.lu.nx : a == 1 ? ns.lu.ny : ns.lu.nz;
                int64_t dst[3], src[3], ext[3];
                for (int b = 0; b < 3; ++b) {
                    if (b == a) {
                        dst[b] = dir < 0 ? -D : n[b];
                        src[b] = dir < 0 ? nn - D : 0;
                        ext[b] = D;
                    } else if (b < a) {  // axes exchanged in an earlier phase: include their ghosts
                        const int64_t gh = b == 0 ? X : D;
                        dst[b] = src[b] = -gh;
                        ext[b] = n[b] + 2 * gh;
                    } else {
                        dst[b] = src[b] = 0;
                        ext[b] = n[b];
                    }
                }
                CopyBox bx{};
                bx.dst_grid = static_cast<int>(i);
                bx.src_grid = ni;
                bx.dst_off = byte_off(s.lu, dst[0], dst[1], dst[2]);
                bx.src_off = byte_off(ns.lu, src[0], src[1], src[2]);
                bx.ex = ext[0];
                bx.ey = ext[1];
                bx.ez = ext[2];
                if (a == 0)
                    widen_x_face(bx, s.lu, ns.lu, dir, D);
                if (bx.ex * bx.ey * bx.ez >= (int64_t(1) << 31))
                    return fail(GBST_EINVAL, "a halo face of %lld cells is too large (limit 2^31 - 1)",
                                static_cast<long long>(bx.ex * bx.ey * bx.ez));
                ph[a].push_back(bx);
            }
    }
    std::vector<CopyBox> all;
    for (int a = 0; a < 3; ++a) {
        h->deep_n[a] = static_cast<int>(ph[a].size());
        h->deep_blocks[a] = halo_copy_blocks(ph[a].data(), h->deep_n[a]);
        all.insert(all.end(), ph[a].begin(), ph[a].end());
    }
    if (!all.empty()) {
        h->ddeep = static_cast<CopyBox *>(dalloc(h, all.size() * sizeof(CopyBox)));
        if (!h->ddeep)
            return fail(GBST_ENOMEM, "halo copy list");
        GBST_CUDA(cudaMemcpyAsync(h->ddeep, all.data(), all.size() * sizeof(CopyBox), cudaMemcpyHostToDevice,
                                  h->stream));
    }
    return GBST_OK;
}

gbst_status build_copies(gbst_handle h)
{
    std::vector<CopyBox> boxes;
    const int R = h->R;
    if (h->subs.size() > 1) {
        auto index_of = [&](const int c[3]) {
            return (c[2] * h->decomp[1] + c[1]) * h->decomp[0] + c[0];
        };
        for (size_t i = 0; i < h->subs.size(); ++i) {
            const Sub &s = h->subs[i];
            for (const Exch &e : exchanges(s, h->decomp, h->ndim, R)) {
                int nc[3] = {s.c[0] + e.to[0], s.c[1] + e.to[1], s.c[2] + e.to[2]};
                const int ni = index_of(nc);
                const Sub &ns = h->subs[ni];
                // the neighbour's exchange that points back at us gives its send region
                const int back[3] = {-e.to[0], -e.to[1], -e.to[2]};
                bool found = false;
                for (const Exch &f : exchanges(ns, h->decomp, h->ndim, R)) {
                    if (f.to[0] != back[0] || f.to[1] != back[1] || f.to[2] != back[2])
                        continue;
                    CopyBox b{};
                    b.dst_grid = static_cast<int>(i);
                    b.src_grid = ni;
                    b.dst_off = byte_off(s.lu, e.at[0], e.at[1], e.at[2]);
                    b.src_off = byte_off(ns.lu, f.at[0] + f.off[0], f.at[1] + f.off[1], f.at[2] + f.off[2]);
                    b.ex = e.size[0];
                    b.ey = e.size[1];
                    b.ez = e.size[2];
                    if (e.to[0] != 0)
                        widen_x_face(b, s.lu, ns.lu, e.to[0], R);
                    boxes.push_back(b);
                    found = true;
                }
                if (!found)
                    return fail(GBST_EINVAL, "internal: unmatched exchange");
            }
        }
    } else if (h->d.bc == GBST_BC_PERIODIC) {
        const Sub &s = h->subs[0];
        const int64_t n[3] = {s.lu.nx, s.lu.ny, s.lu.nz};
        for (int a = 0; a < h->ndim; ++a)
            for (int side = 0; side < 2; ++side) {
                int64_t dst[3] = {0, 0, 0}, src[3] = {0, 0, 0}, ext[3] = {n[0], n[1], n[2]};
                dst[a] = side == 0 ? -R : n[a];
                src[a] = side == 0 ? n[a] - R : 0;
                ext[a] = R;
                CopyBox b{};
                b.dst_grid = b.src_grid = 0;
                b.dst_off = byte_off(s.lu, dst[0], dst[1], dst[2]);
                b.src_off = byte_off(s.lu, src[0], src[1], src[2]);
                b.ex = ext[0];
                b.ey = ext[1];
                b.ez = ext[2];
                if (a == 0)
                    widen_x_face(b, s.lu, s.lu, side == 0 ? -1 : 1, R);
                boxes.push_back(b);
            }
    }
    h->nboxes = static_cast<int>(boxes.size());
    h->max_box_elems = 0;
    for (const CopyBox &b : boxes)
        h->max_box_elems = std::max(h->max_box_elems, b.ex * b.ey * b.ez);
    if (h->max_box_elems >= (int64_t(1) << 31))
        return fail(GBST_EINVAL, "a halo face of %lld cells is too large (limit 2^31 - 1)",
                    static_cast<long long>(h->max_box_elems));
    h->copy_blocks = halo_copy_blocks(boxes.data(), static_cast<int>(boxes.size()));
    if (!boxes.empty()) {
        h->dboxes = static_cast<CopyBox *>(dalloc(h, boxes.size() * sizeof(CopyBox)));
        if (!h->dboxes)
            return fail(GBST_ENOMEM, "halo copy list");
        GBST_CUDA(cudaMemcpyAsync(h->dboxes, boxes.data(), boxes.size() * sizeof(CopyBox), cudaMemcpyHostToDevice,
                                  h->stream));
    }
    return h->deep ? build_deep_copies(h) : GBST_OK;
}

SweepArgs sweep_args(gbst_handle h, int parity, const float *srcval)
{
    SweepArgs a{};
    a.grids = h->dgrids;
    a.units = h->dunits;
    a.nunits = h->plan.nunits;
    a.parity = parity;
    a.ndim = h->ndim;
    // integer weights (exact in FP32, so the star of a constant is exactly 0); the common
    // denominator is in the coefficients (heat_a, the coupling matrix) or, for the wave,
    // in lscale, which multiplies the sum before kappa
    a.wc = static_cast<float>(h->ndim * h->wint[0]);
    for (int m = 1; m <= h->R; ++m)
        a.w[m] = static_cast<float>(h->wint[m]);
    a.lscale = static_cast<float>(1.0 / h->wscale);
    a.srcval = srcval;
    a.err = h->derr;
    a.nsteps = 1;
    a.ngrids = static_cast<int>(h->subs.size());
    a.barrier = h->dbarrier;
    a.barrier_extra = h->barrier_extra;
    // the dynamic-assignment counters share the grid-barrier buffer (zeroed at creation)
    a.dyn = h->plan.dyn ? h->dbarrier + kDynCounterOffset : nullptr;
    for (int k = 0; k < 16; ++k)
        a.coupling[k] = h->coupling[k];
    return a;
}

// Enqueue one sweep launch (halo copies + sweep) at the given parity: one time
// step, or two with a temporally blocked plan unless `single`.
gbst_status enqueue_step(gbst_handle h, int parity, const float *srcval, int prof_index, bool single = false)
{
    if (h->plan.stream && h->plan.overlap && h->nboxes > 0) {
        // The halo copies run on a second stream while the units that read no
        // exchanged ghost cell sweep; the other units sweep once the copies are done.
        // (The copies write ghosts of u^n and read neighbours' interior u^n; the sweep
        // reads u^n and writes the other buffer.)
        if (!h->side) {
            GBST_CUDA(cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking));
            GBST_CUDA(cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
            GBST_CUDA(cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming));
        }
        GBST_CUDA(cudaEventRecord(h->ev_fork, h->stream));
        GBST_CUDA(cudaStreamWaitEvent(h->side, h->ev_fork, 0));
        cudaError_t e =
            launch_halo_copies(h->dgrids, h->dboxes, h->nboxes, parity, h->es, h->copy_blocks, h->side);
        if (e != cudaSuccess)
            return fail(GBST_ECUDA, "halo copy launch: %s", cudaGetErrorString(e));
        GBST_CUDA(cudaEventRecord(h->ev_join, h->side));
        SweepArgs a = sweep_args(h, parity, srcval);
        if (prof_index >= 0)
            GBST_CUDA(cudaEventRecordWithFlags(h->prof_ev[2 * prof_index], h->stream, cudaEventRecordExternal));
        const int nint = h->plan.nint, nlate = h->plan.nunits - h->plan.nint;
        a.nunits = nint;
        e = launch_stream_sweep(h->plan.var, a, std::min(h->plan.ctas, nint), h->plan.smem, h->stream);
        if (e != cudaSuccess)
            return fail(GBST_ECUDA, "sweep launch: %s", cudaGetErrorString(e));
        GBST_CUDA(cudaStreamWaitEvent(h->stream, h->ev_join, 0));
        a.units = h->dunits + nint;
        a.nunits = nlate;
        e = launch_stream_sweep(h->plan.var, a, std::min(h->plan.ctas, nlate), h->plan.smem, h->stream);
        if (e != cudaSuccess)
            return fail(GBST_ECUDA, "sweep launch: %s", cudaGetErrorString(e));
        if (prof_index >= 0)
            GBST_CUDA(cudaEventRecordWithFlags(h->prof_ev[2 * prof_index + 1], h->stream,
                                               cudaEventRecordExternal));
        return GBST_OK;
    }
    if (h->deep && h->plan.stream && h->plan.var.tb == 2) {
        // two steps follow: faces 2r deep and the edges, in three ordered phases
        const CopyBox *b = h->ddeep;
        for (int a = 0; a < 3; ++a) {
            const cudaError_t e =
                launch_halo_copies(h->dgrids, b, h->deep_n[a], parity, h->es, h->deep_blocks[a], h->stream);
            if (e != cudaSuccess)
                return fail(GBST_ECUDA, "halo copy launch: %s", cudaGetErrorString(e));
            b += h->deep_n[a];
        }
    } else if (h->nboxes > 0) {
        cudaError_t e =
            launch_halo_copies(h->dgrids, h->dboxes, h->nboxes, parity, h->es, h->copy_blocks, h->stream);
        if (e != cudaSuccess)
            return fail(GBST_ECUDA, "halo copy launch: %s", cudaGetErrorString(e));
    }
    SweepArgs a = sweep_args(h, parity, srcval);
    a.tb_single = single ? 1 : 0;
    if (prof_index >= 0)
        GBST_CUDA(cudaEventRecordWithFlags(h->prof_ev[2 * prof_index], h->stream,
                                           cudaEventRecordExternal));
    cudaError_t e;
    if (h->plan.stream)
        e = launch_stream_sweep(h->plan.var, a, h->plan.ctas, h->plan.smem, h->stream);
    else
        e = launch_simple_sweep(h->R, h->d.eq, h->d.storage, a, static_cast<int>(h->subs.size()), h->max_points,
                                h->stream);
    if (e != cudaSuccess)
        return fail(GBST_ECUDA, "sweep launch: %s", cudaGetErrorString(e));
    if (prof_index >= 0)
        GBST_CUDA(cudaEventRecordWithFlags(h->prof_ev[2 * prof_index + 1], h->stream,
                                           cudaEventRecordExternal));
    if (h->closure) {
        // u^{n+1} += closure(u^{n+1}, u^n, c_norm): gather both levels dense, run the
        // network, add the correction back into the padded field
        const Sub &sb = h->subs[0];
        const GridDev &g = h->hgrids[0];
        XferArgs x{};
        x.storage = h->d.storage;
        x.pitch = sb.lu.pitch;
        x.rows = sb.lu.rows;
        x.origin = sb.lu.origin;
        x.nx = sb.lu.nx;
        x.ny = sb.lu.ny;
        x.nz = sb.lu.nz;
        x.gnx = sb.lu.nx;
        x.gny = sb.lu.ny;
        x.dense_dtype = GBST_F32;
        x.padded = g.buf[1 - parity];
        x.dense = h->cl_up;
        GBST_CUDA(launch_gather(x, h->stream));
        x.padded = g.buf[parity];
        x.dense = h->cl_un;
        GBST_CUDA(launch_gather(x, h->stream));
        gbst_status cs = closure_forward(h->closure, h->cl_up, h->cl_un, h->cl_cn, sb.lu.nx, sb.lu.ny, sb.lu.nz,
                                         h->cl_corr);
        if (cs != GBST_OK)
            return cs;
        x.padded = g.buf[1 - parity];
        x.dense = h->cl_corr;
        GBST_CUDA(launch_scatter_add(x, h->stream));
    }
    return GBST_OK;
}

// Enqueue a whole run as one persistent launch (grid-wide barriers between steps).
gbst_status enqueue_persistent(gbst_handle h, int64_t nsteps, int parity, const float *srcval, bool prof)
{
    GBST_CUDA(cudaMemsetAsync(h->dbarrier, 0, sizeof(unsigned int), h->stream));
    SweepArgs a = sweep_args(h, parity, srcval);
    a.nsteps = static_cast<int>(nsteps);
    if (prof)
        GBST_CUDA(cudaEventRecordWithFlags(h->prof_ev[0], h->stream, cudaEventRecordExternal));
    const cudaError_t e = launch_stream_sweep(h->plan.var, a, h->plan.ctas, h->plan.smem, h->stream, true);
    if (e != cudaSuccess)
        return fail(GBST_ECUDA, "persistent sweep launch: %s", cudaGetErrorString(e));
    if (prof)
        GBST_CUDA(cudaEventRecordWithFlags(h->prof_ev[1], h->stream, cudaEventRecordExternal));
    return GBST_OK;
}

double ricker(double t, double f0, double t0)
{
    const double a = M_PI * f0 * (t - t0);
    const double a2 = a * a;
    return (1.0 - 2.0 * a2) * std::exp(-a2);
}

gbst_status ensure_src_capacity(gbst_handle h, int64_t nsteps)
{
    const int64_t ns = static_cast<int64_t>(h->subs.size());
    if (nsteps <= h->src_cap)
        return GBST_OK;
    int64_t cap = std::max<int64_t>(nsteps, 64);
    if (h->dsrc)
        dfree(h, h->dsrc);
    if (h->hsrc)
        cudaFreeHost(h->hsrc);
    h->hsrc = nullptr;
    h->dsrc = static_cast<float *>(dalloc(h, cap * ns * sizeof(float)));
    if (!h->dsrc)
        return fail(GBST_ENOMEM, "source table");
    GBST_CUDA(cudaMallocHost(&h->hsrc, cap * ns * sizeof(float)));
    h->src_cap = cap;
    destroy_graphs(h);  // graphs reference the table address
    return GBST_OK;
}

gbst_status read_kappa_at_source(gbst_handle h)
{
    GBST_CUDA(cudaStreamSynchronize(h->stream));
    for (size_t i = 0; i < h->subs.size(); ++i) {
        Sub &s = h->subs[i];
        if (!s.src_on)
            continue;
        const int64_t k = h->ndim == 3 ? s.src_local[2] : 0;
        const int64_t idx = s.lk.origin + (k * s.lk.rows + s.src_local[1]) * s.lk.pitch + s.src_local[0];
        float v = 0.f;
        GBST_CUDA(cudaMemcpy(&v, h->hgrids[i].kappa + idx, sizeof(float), cudaMemcpyDeviceToHost));
        s.kappa_src = v;
    }
    return GBST_OK;
}

// Validate one grid description; dims receives the interior sizes (z = 1 in 2D).
gbst_status validate_desc(const gbst_desc &d, int64_t dims[3], int decomp[3])
{
    if (d.ndim != 2 && d.ndim != 3)
        return fail(GBST_EINVAL, "ndim must be 2 or 3");
    if (d.space_order != 2 && d.space_order != 4 && d.space_order != 8)
        return fail(GBST_EINVAL, "space_order must be 2, 4 or 8");
    if (d.eq != GBST_HEAT && d.eq != GBST_WAVE)
        return fail(GBST_EINVAL, "eq must be GBST_HEAT or GBST_WAVE");
    if (d.bc != GBST_BC_ZERO && d.bc != GBST_BC_PERIODIC)
        return fail(GBST_EINVAL, "bc must be GBST_BC_ZERO or GBST_BC_PERIODIC");
    if (d.storage != GBST_F32 && d.storage != GBST_BF16)
        return fail(GBST_EINVAL, "storage must be GBST_F32 or GBST_BF16");
    if (d.kernel < GBST_KERNEL_AUTO || d.kernel > GBST_KERNEL_SIMPLE)
        return fail(GBST_EINVAL, "kernel must be GBST_KERNEL_AUTO, _STREAM or _SIMPLE");
    if (d.temporal_block < 0 || d.temporal_block > 2)
        return fail(GBST_EINVAL, "temporal_block must be 0 (automatic), 1 (off) or 2");
    const int R = d.space_order / 2;
    dims[0] = d.dims[0];
    dims[1] = d.dims[1];
    dims[2] = d.ndim == 3 ? d.dims[2] : 1;
    for (int a = 0; a < d.ndim; ++a)
        if (dims[a] < 1 || dims[a] > (int64_t(1) << 30))
            return fail(GBST_EINVAL, "dims[%d] = %lld out of range", a, static_cast<long long>(dims[a]));
    for (int a = 0; a < 3; ++a) {
        decomp[a] = d.decomp[a] <= 0 ? 1 : d.decomp[a];
        if (a >= d.ndim && decomp[a] != 1)
            return fail(GBST_EINVAL, "decomp[%d] must be 1 for a %dD grid", a, d.ndim);
        if (decomp[a] > dims[a])
            return fail(GBST_EINVAL, "decomp[%d] larger than the grid", a);
    }
    const bool decomposed = decomp[0] * decomp[1] * decomp[2] > 1;
    if (decomposed && d.bc == GBST_BC_PERIODIC)
        return fail(GBST_ENOTSUP, "periodic boundaries are not supported in decomposition mode");
    if (d.bc == GBST_BC_PERIODIC)
        for (int a = 0; a < d.ndim; ++a)
            if (dims[a] < R)
                return fail(GBST_EINVAL, "periodic boundaries need at least r points per axis");
    if (d.h <= 0.0 || d.dt <= 0.0)
        return fail(GBST_EINVAL, "h and dt must be positive");
    return GBST_OK;
}

gbst_status destroy_handle(gbst_handle h);

// Create a handle from n descriptions: n == 1 is a single (possibly decomposed)
// grid; n > 1 a batch of independent grids sharing dimensionality, order,
// equation, storage and weights (each with its own sizes, step and spacing).
// Largest singular value of a small square matrix (n <= 4): Jacobi sweeps on B^T B.
double max_singular_value(const double *B, int n)
{
    double M[4][4] = {{0}};
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j)
            for (int k = 0; k < n; ++k)
                M[i][j] += B[k * n + i] * B[k * n + j];
    for (int sweep = 0; sweep < 50; ++sweep) {
        double off = 0.0;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q)
                off += M[p][q] * M[p][q];
        if (off < 1e-30)
            break;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) {
                if (std::fabs(M[p][q]) < 1e-300)
                    continue;
                const double th = 0.5 * std::atan2(2.0 * M[p][q], M[q][q] - M[p][p]);
                const double c = std::cos(th), sn = std::sin(th);
                for (int k = 0; k < n; ++k) {  // rotate columns p, q
                    const double mkp = M[k][p], mkq = M[k][q];
                    M[k][p] = c * mkp - sn * mkq;
                    M[k][q] = sn * mkp + c * mkq;
                }
                for (int k = 0; k < n; ++k) {  // rotate rows p, q
                    const double mpk = M[p][k], mqk = M[q][k];
                    M[p][k] = c * mpk - sn * mqk;
                    M[q][k] = sn * mpk + c * mqk;
                }
            }
    }
    double mx = 0.0;
    for (int i = 0; i < n; ++i)
        mx = std::max(mx, M[i][i]);
    return std::sqrt(std::max(mx, 0.0));
}

// Stability of u <- u + A L(u) (sufficient): |I + lambda A|_2 <= 1 for every
// symbol value lambda in [-ndim S, 0] (exact for symmetric A and for A = a I).
// Writes the weights w[0..R] as integers wint over the smallest common denominator
// *scale (w = wint / scale) when one up to 10^6 exists with integers below 2^22 (exact in
// FP32, and 2 ndim |wint[0]| too); else wint = w, *scale = 1.
void integer_weights(int R, const double *w, double *wint, double *scale)
{
    for (int m = 0; m <= R; ++m)
        wint[m] = w[m];
    *scale = 1.0;
    for (int S = 1; S <= 1000000; ++S) {
        bool ok = true;
        for (int m = 0; m <= R && ok; ++m) {
            const double v = w[m] * S;
            ok = std::fabs(v - std::nearbyint(v)) <= 1e-9 * std::max(1.0, std::fabs(v)) && std::fabs(v) < 4194304.0;
        }
        if (ok) {
            for (int m = 0; m <= R; ++m)
                wint[m] = std::nearbyint(w[m] * S);
            *scale = S;
            return;
        }
    }
}

bool system_stable(const double *A, int n, int ndim, double S)
{
    double B[16];
    for (int t = 0; t <= 512; ++t) {
        const double lam = -ndim * S * t / 512.0;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j)
                B[i * n + j] = (i == j ? 1.0 : 0.0) + lam * A[i * n + j];
        if (max_singular_value(B, n) > 1.0 + 1e-9)
            return false;
    }
    return true;
}

gbst_status create_handle(const gbst_desc *descs, int n, bool batch, gbst_handle *out, int nfields = 0,
                          const double *coupling = nullptr)
{
    if (!descs || !out || n < 1)
        return fail(GBST_EINVAL, "null descriptions or handle, or n < 1");
    *out = nullptr;
    const gbst_desc &d = descs[0];
    int64_t dims0[3];
    int decomp[3];
    gbst_status st = validate_desc(d, dims0, decomp);
    if (st != GBST_OK)
        return st;
    const int R = d.space_order / 2;
    for (int i = 1; i < n; ++i) {
        int64_t di[3];
        int dc[3];
        st = validate_desc(descs[i], di, dc);
        if (st != GBST_OK)
            return st;
        const gbst_desc &e = descs[i];
        if (e.ndim != d.ndim || e.space_order != d.space_order || e.eq != d.eq || e.storage != d.storage ||
            e.bc != d.bc || e.kernel != d.kernel)
            return fail(GBST_EINVAL, "batch member %d differs in ndim/order/equation/storage/bc/kernel", i);
    }
    if (batch) {
        for (int i = 0; i < n; ++i) {
            const gbst_desc &e = descs[i];
            if (e.bc != GBST_BC_ZERO)
                return fail(GBST_ENOTSUP, "batch members need zero (Dirichlet) halos");
            for (int a = 0; a < 3; ++a)
                if (e.decomp[a] > 1)
                    return fail(GBST_ENOTSUP, "batch members cannot be decomposed");
        }
    }

    gbst_handle h = new (std::nothrow) gbst_grid_s;
    if (!h)
        return fail(GBST_ENOMEM, "handle");
    h->d = d;
    h->d.coeffs = nullptr;
    h->ndim = d.ndim;
    h->R = R;
    h->es = d.storage == GBST_BF16 ? 2 : 4;
    h->batch = batch;
    h->members = n;
    for (int a = 0; a < 3; ++a)
        h->decomp[a] = batch ? 1 : decomp[a];
    if (d.coeffs)
        for (int m = 0; m <= R; ++m)
            h->w[m] = d.coeffs[m];
    else
        central_weights(R, h->w);
    h->S = symbol_max(R, h->w);
    integer_weights(R, h->w, h->wint, &h->wscale);
    h->stream = static_cast<cudaStream_t>(d.stream);
    h->mem.s = h->stream;
    if (d.allocator) {
        if (!d.allocator->alloc || !d.allocator->release) {
            delete h;
            return fail(GBST_EINVAL, "allocator needs alloc and release");
        }
        h->mem.a = *d.allocator;
        h->mem.custom = true;
    }
    if (nfields > 0) {
        h->nf = nfields;
        for (int k = 0; k < nfields * nfields; ++k)
            h->coupling[k] = static_cast<float>(coupling[k] / h->wscale);
        if (!d.allow_unstable && !system_stable(coupling, nfields, h->ndim, h->S)) {
            delete h;
            return fail(GBST_EUNSTABLE, "coupling matrix: |I + lambda A| > 1 for a symbol value lambda of the stencil");
        }
    } else {
        for (int i = 0; i < n; ++i) {
            const gbst_desc &e = descs[i];
            const double a = e.alpha * e.dt / (e.h * e.h);
            if (e.eq == GBST_HEAT && !e.allow_unstable && a * h->ndim * h->S > 2.0 * (1.0 + 1e-12)) {
                delete h;
                return fail(GBST_EUNSTABLE, "heat step a*ndim*S = %g exceeds 2 (von Neumann limit)",
                            a * d.ndim * h->S);
            }
        }
    }

    // decomposed heat grids that two-step blocking can sweep (radius 1 or 2: the
    // blocked variants) keep ghost regions 2r deep; see build_copies
    h->deep = !batch && h->nf == 1 && h->decomp[0] * h->decomp[1] * h->decomp[2] > 1 && d.eq == GBST_HEAT &&
              d.storage == GBST_F32 && d.ndim == 3 && d.bc == GBST_BC_ZERO && d.temporal_block != 1 &&
              d.kernel != GBST_KERNEL_SIMPLE && R <= 2;
    const int ghost = h->deep ? 2 * R : R;

    auto bail = [&](gbst_status code) {
        destroy_handle(h);
        return code;
    };

    // subdomains: equal slicing, the first n mod D parts one larger
    auto split = [](int64_t len, int parts, int i, int64_t *start) {
        const int64_t base = len / parts, rem = len % parts;
        *start = i * base + std::min<int64_t>(i, rem);
        return base + (i < rem ? 1 : 0);
    };
    const int px = px_of(d.storage);
    for (int mi = 0; mi < n; ++mi) {
        const gbst_desc &e = descs[mi];
        int64_t dims[3];
        int dc[3];
        validate_desc(e, dims, dc);
        const int *dd = h->decomp;  // all ones for a batch
        for (int cz = 0; cz < dd[2]; ++cz)
            for (int cy = 0; cy < dd[1]; ++cy)
                for (int cx = 0; cx < dd[0]; ++cx) {
                    Sub s{};
                    s.c[0] = cx;
                    s.c[1] = cy;
                    s.c[2] = cz;
                    s.member = mi;
                    s.dt = e.dt;
                    s.h = e.h;
                    s.alpha = e.alpha;
                    for (int a = 0; a < 3; ++a)
                        s.dense[a] = dims[a];
                    int64_t nn[3];
                    nn[0] = split(dims[0], dd[0], cx, &s.g0[0]);
                    nn[1] = split(dims[1], dd[1], cy, &s.g0[1]);
                    nn[2] = split(dims[2], dd[2], cz, &s.g0[2]);
                    // x ghosts of 128 bytes for wide rows (interior rows start on a
                    // 128-byte line: 1.47 against 1.50 ms per order-8 sweep at 1024^3);
                    // one 16-byte chunk for narrow rows, where the wider row pitch cost
                    // more than it saved (64 grids of 96-256 points per axis: 353
                    // against 388 GPoints/s)
                    const bool wide = nn[0] * h->es >= kWideRowBytes;
                    s.lu = make_layout(d.ndim, nn[0], nn[1], nn[2], ghost, h->es, (wide ? kGhostBytesX : 16) / h->es);
                    s.lk = make_layout(d.ndim, nn[0], nn[1], nn[2], R, 4, wide ? kGhostBytesX / 4 : px);
                    h->subs.push_back(s);
                    h->max_points = std::max(h->max_points, nn[0] * nn[1] * nn[2]);
                }
    }
    // a two-step exchange reaches 2r cells into each neighbour: every subdomain needs that many
    for (const Sub &sb : h->subs) {
        const int64_t ext[3] = {sb.lu.nx, sb.lu.ny, sb.lu.nz};
        for (int a = 0; a < 3; ++a)
            if (h->decomp[a] > 1 && ext[a] < 2 * R)
                h->deep = false;  // (the layouts keep their deep ghosts; only single steps run)
    }
    const size_t ns = h->subs.size();
    h->hgrids.assign(ns, GridDev{});
    for (size_t i = 0; i < ns; ++i) {
        const Sub &s = h->subs[i];
        GridDev &g = h->hgrids[i];
        for (int b = 0; b < 2; ++b) {
            g.buf[b] = dalloc(h, s.lu.bytes);
            if (!g.buf[b]) {
                fail(GBST_ENOMEM, "field allocation of %zu bytes", s.lu.bytes);
                return bail(GBST_ENOMEM);
            }
            if (cudaMemsetAsync(g.buf[b], 0, s.lu.bytes, h->stream) != cudaSuccess) {
                fail(GBST_ECUDA, "memset of a field");
                return bail(GBST_ECUDA);
            }
        }
        if (d.eq == GBST_WAVE) {
            g.kappa = static_cast<float *>(dalloc(h, s.lk.bytes));
            if (!g.kappa) {
                fail(GBST_ENOMEM, "kappa allocation");
                return bail(GBST_ENOMEM);
            }
            if (cudaMemsetAsync(g.kappa, 0, s.lk.bytes, h->stream) != cudaSuccess) {
                fail(GBST_ECUDA, "memset of kappa");
                return bail(GBST_ECUDA);
            }
        }
        g.nx = s.lu.nx;
        g.ny = s.lu.ny;
        g.nz = s.lu.nz;
        g.pitch = s.lu.pitch;
        g.rows = s.lu.rows;
        g.origin = s.lu.origin;
        g.kpitch = s.lk.pitch;
        g.krows = s.lk.rows;
        g.korigin = s.lk.origin;
        g.heat_a = static_cast<float>(s.alpha * s.dt / (s.h * s.h) / h->wscale);
        g.ghost = s.lu.r;
        g.face_int = 0;
        for (int a = 0; a < d.ndim; ++a) {
            if (s.c[a] > 0)
                g.face_int |= 1 << (2 * a);
            if (s.c[a] + 1 < h->decomp[a])
                g.face_int |= 2 << (2 * a);
        }
    }
    h->dgrids = static_cast<GridDev *>(dalloc(h, ns * sizeof(GridDev)));
    h->derr = static_cast<int *>(dalloc(h, 256));
    h->dbarrier = static_cast<unsigned int *>(dalloc(h, 256));
    h->red_blocks_per_grid = std::max(1, reduce_blocks_for(h->max_points) / static_cast<int>(std::min<size_t>(ns, 8)));
    h->dpartials = static_cast<double *>(dalloc(h, ns * h->red_blocks_per_grid * sizeof(double)));
    h->dred_out = static_cast<double *>(dalloc(h, 256));
    h->dred_grids = static_cast<ReduceGrid *>(dalloc(h, ns * sizeof(ReduceGrid)));
    if (!h->dgrids || !h->derr || !h->dbarrier || !h->dpartials || !h->dred_out || !h->dred_grids) {
        fail(GBST_ENOMEM, "metadata allocation");
        return bail(GBST_ENOMEM);
    }
    if (cudaMemsetAsync(h->derr, 0, 256, h->stream) != cudaSuccess ||
        cudaMemsetAsync(h->dbarrier, 0, 256, h->stream) != cudaSuccess) {
        fail(GBST_ECUDA, "memset of the error word");
        return bail(GBST_ECUDA);
    }
    st = build_copies(h);
    if (st != GBST_OK)
        return bail(st);
    TunedPlan tp{};
    StreamVariant cv;
    // (a cached plan is used only if it honours an explicit request for two-step sweeps)
    if (d.tile == 0 && d.kernel != GBST_KERNEL_SIMPLE && tune_cache_find(h, &tp) &&
        stream_variant_get(tp.variant, &cv) && variant_matches(h, cv) &&
        !(d.temporal_block == 2 && tb_allowed(h) && cv.tb != 2)) {
        h->dyn_pref = tp.dyn;
        st = build_plan(h, tp.variant, tp.txt, tp.zchunks, tp.ctas);
    } else {
        st = build_plan(h, d.tile > 0 ? d.tile - 1 : -1, 0, 0, 0);
    }
    if (st != GBST_OK)
        return bail(st);
    *out = h;
    return GBST_OK;
}

gbst_status destroy_handle(gbst_handle h)
{
    if (!h)
        return GBST_OK;
    cudaStreamSynchronize(h->stream);
    destroy_graphs(h);
    if (h->side) {
        cudaStreamSynchronize(h->side);
        cudaStreamDestroy(h->side);
    }
    if (h->ev_fork)
        cudaEventDestroy(h->ev_fork);
    if (h->ev_join)
        cudaEventDestroy(h->ev_join);
    for (cudaEvent_t e : h->prof_ev)
        cudaEventDestroy(e);
    if (h->src_ev)
        cudaEventDestroy(h->src_ev);
    if (h->hsrc)
        cudaFreeHost(h->hsrc);
    for (DevMem &m : h->owned)
        h->mem.release(m.p, m.bytes);
    h->owned.clear();
    delete h;
    return GBST_OK;
}

// Copy one member's dense field in (to_dev) or out.
gbst_status transfer(gbst_handle h, int member, int field, void *user, int dtype, int on_device, bool to_dev,
                     bool async = false)
{
    gbst_status st = check_handle(h);
    if (st != GBST_OK)
        return st;
    if (!user)
        return fail(GBST_EINVAL, "null buffer");
    if (member < 0 || member >= h->members)
        return fail(GBST_EINVAL, "grid index %d out of range [0, %d)", member, h->members);
    if (dtype != GBST_F32 && dtype != GBST_F64 && dtype != GBST_BF16)
        return fail(GBST_EINVAL, "dtype must be GBST_F32, GBST_F64 or GBST_BF16");
    if (field != GBST_U && field != GBST_U_PREV && field != GBST_VEL)
        return fail(GBST_EINVAL, "unknown field %d", field);
    if (h->d.eq == GBST_HEAT && field != GBST_U)
        return fail(GBST_EINVAL, "heat grids have only the field GBST_U");
    const size_t esz = dtype == GBST_F64 ? 8 : dtype == GBST_F32 ? 4 : 2;
    size_t n = 0;
    for (const Sub &s : h->subs)
        if (s.member == member) {
            n = static_cast<size_t>(s.dense[0] * s.dense[1] * s.dense[2]);
            break;
        }
    void *dense = user;
    void *staging = nullptr;
    if (async && !on_device) {
        // host memory moves by the copy engines through a device staging buffer (no SMs
        // held while the host link is busy); only page-locked memory copies asynchronously
        cudaPointerAttributes pa{};
        const bool pinned = cudaPointerGetAttributes(&pa, user) == cudaSuccess && pa.type == cudaMemoryTypeHost;
        cudaGetLastError();
        if (!pinned)
            return fail(GBST_EINVAL, "asynchronous transfers need device memory or page-locked host memory");
    }
    if (async && field == GBST_VEL)
        return fail(GBST_EINVAL, "GBST_VEL is transferred synchronously (its stability check reads it back)");
    if (async && !on_device && dtype == h->d.storage) {
        // Page-locked host memory in the storage type and a member of one subdomain: the
        // copy engines move the interior straight between the dense host array and the
        // padded field (a pitched 3D copy: no staging buffer, no transfer kernel on the SMs,
        // measured as fast as a contiguous copy of the same bytes).
        int nsub = 0;
        size_t si = 0;
        for (size_t i = 0; i < h->subs.size(); ++i)
            if (h->subs[i].member == member) {
                ++nsub;
                si = i;
            }
        if (nsub == 1) {
            const Layout &L = h->subs[si].lu;
            void *padded = h->hgrids[si].buf[field == GBST_U ? h->parity : 1 - h->parity];
            const size_t row = static_cast<size_t>(L.nx) * esz;
            cudaMemcpy3DParms p{};
            const cudaPitchedPtr dp = make_cudaPitchedPtr(padded, static_cast<size_t>(L.pitch) * L.es,
                                                          static_cast<size_t>(L.pitch) * L.es,
                                                          static_cast<size_t>(L.rows));
            const cudaPitchedPtr hp = make_cudaPitchedPtr(user, row, row, static_cast<size_t>(L.ny));
            const cudaPos interior = make_cudaPos(static_cast<size_t>(L.G) * L.es, static_cast<size_t>(L.r),
                                                  static_cast<size_t>(L.rz));
            p.extent = make_cudaExtent(row, static_cast<size_t>(L.ny), static_cast<size_t>(L.nz));
            if (to_dev) {
                p.srcPtr = hp;
                p.dstPtr = dp;
                p.dstPos = interior;
                p.kind = cudaMemcpyHostToDevice;
            } else {
                p.srcPtr = dp;
                p.srcPos = interior;
                p.dstPtr = hp;
                p.kind = cudaMemcpyDeviceToHost;
            }
            GBST_CUDA(cudaMemcpy3DAsync(&p, h->stream));
            return GBST_OK;  // errors surface at the next synchronising call
        }
    }
    if (!on_device) {
        staging = h->mem.alloc(n * esz);
        if (!staging)
            return fail(GBST_ENOMEM, "staging buffer of %zu bytes", n * esz);
        dense = staging;
        if (to_dev) {
            cudaError_t e = cudaMemcpyAsync(staging, user, n * esz, cudaMemcpyHostToDevice, h->stream);
            if (e != cudaSuccess) {
                h->mem.release(staging, n * esz);
                return fail(GBST_ECUDA, "host-to-device copy: %s", cudaGetErrorString(e));
            }
        }
    }
    for (size_t i = 0; i < h->subs.size(); ++i) {
        const Sub &s = h->subs[i];
        if (s.member != member)
            continue;
        const GridDev &g = h->hgrids[i];
        XferArgs x{};
        const bool kap = field == GBST_VEL;
        const Layout &L = kap ? s.lk : s.lu;
        x.padded = kap ? static_cast<void *>(g.kappa) : g.buf[field == GBST_U ? h->parity : 1 - h->parity];
        x.storage = kap ? GBST_F32 : h->d.storage;
        x.pitch = L.pitch;
        x.rows = L.rows;
        x.origin = L.origin;
        x.nx = L.nx;
        x.ny = L.ny;
        x.nz = L.nz;
        x.gx = s.g0[0];
        x.gy = s.g0[1];
        x.gz = s.g0[2];
        x.gnx = s.dense[0];
        x.gny = s.dense[1];
        x.dense = dense;
        x.dense_dtype = dtype;
        x.scale_sq = (kap && to_dev) ? (s.dt * s.dt) / (s.h * s.h) : 0.0;
        cudaError_t e = to_dev ? launch_scatter(x, h->stream) : launch_gather(x, h->stream);
        if (e != cudaSuccess) {
            if (staging)
                h->mem.release(staging, n * esz);
            return fail(GBST_ECUDA, "transfer kernel: %s", cudaGetErrorString(e));
        }
    }
    if (!on_device && !to_dev) {
        cudaError_t e = cudaMemcpyAsync(user, staging, n * esz, cudaMemcpyDeviceToHost, h->stream);
        if (e != cudaSuccess) {
            h->mem.release(staging, n * esz);
            return fail(GBST_ECUDA, "device-to-host copy: %s", cudaGetErrorString(e));
        }
    }
    if (async) {
        // the staging buffer returns to the allocator in stream order (the torch
        // caching allocator reuses it only for later work on the same stream)
        if (staging)
            h->mem.release(staging, n * esz);
        return GBST_OK;  // errors surface at the next synchronising call
    }
    st = poll_device_error(h);
    if (staging)
        h->mem.release(staging, n * esz);
    return st;
}

// FP64 reduction over the subdomains of one member (member < 0: all of them).
gbst_status reduce_member(gbst_handle h, int member, int kind, int field_is_kappa, double *out)
{
    std::vector<ReduceGrid> rg;
    int64_t maxp = 0;
    for (size_t i = 0; i < h->subs.size(); ++i) {
        const Sub &s = h->subs[i];
        if (member >= 0 && s.member != member)
            continue;
        const GridDev &g = h->hgrids[i];
        if (field_is_kappa)
            rg.push_back(ReduceGrid{g.kappa, nullptr, nullptr, s.lk.pitch, s.lk.rows, s.lk.origin, 0, 0, 0, s.lk.nx,
                                    s.lk.ny, s.lk.nz});
        else
            rg.push_back(ReduceGrid{g.buf[h->parity], g.buf[1 - h->parity], g.kappa, s.lu.pitch, s.lu.rows,
                                    s.lu.origin, s.lk.pitch, s.lk.rows, s.lk.origin, s.lu.nx, s.lu.ny, s.lu.nz});
        maxp = std::max(maxp, s.lu.nx * s.lu.ny * s.lu.nz);
    }
    const int ng = static_cast<int>(rg.size());
    GBST_CUDA(cudaMemcpyAsync(h->dred_grids, rg.data(), rg.size() * sizeof(ReduceGrid), cudaMemcpyHostToDevice,
                              h->stream));
    const int nb = h->red_blocks_per_grid * ng;
    GBST_CUDA(launch_reduce_partials(kind, field_is_kappa ? GBST_F32 : h->d.storage, h->ndim, h->R, h->w,
                                     h->dred_grids, ng, maxp, h->dpartials, nb, h->stream));
    GBST_CUDA(launch_reduce_final(kind, h->dpartials, nb, h->dred_out, h->stream));
    double v = 0.0;
    GBST_CUDA(cudaMemcpyAsync(&v, h->dred_out, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    gbst_status st = poll_device_error(h);
    if (st != GBST_OK)
        return st;
    *out = v;
    return GBST_OK;
}

gbst_status set_field_member(gbst_handle h, int member, int field, const void *src, int dtype, int on_device)
{
    gbst_status st = transfer(h, member, field, const_cast<void *>(src), dtype, on_device, true);
    if (st != GBST_OK || field != GBST_VEL)
        return st;
    st = read_kappa_at_source(h);
    if (st != GBST_OK)
        return st;
    // stability of the leapfrog scheme: kappa_max * ndim * S <= 4
    double kmax = 0.0;
    st = reduce_member(h, member, GBST_RED_MAXABS, 1, &kmax);
    if (st != GBST_OK)
        return st;
    const bool unstable = kmax * h->ndim * h->S > 4.0 * (1.0 + 1e-9);
    for (Sub &s : h->subs)
        if (s.member == member)
            s.unstable = unstable;
    if (unstable && !h->d.allow_unstable)
        return fail(GBST_EUNSTABLE, "wave step: kappa_max*ndim*S = %g exceeds 4 (CFL limit)", kmax * h->ndim * h->S);
    return GBST_OK;
}

gbst_status set_source_member(gbst_handle h, int member, const int64_t idx[3], double f0_hz, double t0_s,
                              double amp)
{
    gbst_status st = check_handle(h);
    if (st != GBST_OK)
        return st;
    if (h->d.eq != GBST_WAVE)
        return fail(GBST_EINVAL, "sources are only defined for the wave equation");
    if (member < 0 || member >= h->members)
        return fail(GBST_EINVAL, "grid index %d out of range", member);
    for (size_t i = 0; i < h->subs.size(); ++i)
        if (h->subs[i].member == member) {
            h->subs[i].src_on = false;
            h->hgrids[i].has_src = 0;
        }
    if (f0_hz > 0.0) {
        if (!idx)
            return fail(GBST_EINVAL, "null source index");
        bool placed = false;
        for (size_t i = 0; i < h->subs.size(); ++i) {
            Sub &s = h->subs[i];
            if (s.member != member)
                continue;
            const int64_t p[3] = {idx[0], idx[1], h->ndim == 3 ? idx[2] : 0};
            bool in = true;
            for (int a = 0; a < 3; ++a) {
                if (p[a] < 0 || p[a] >= s.dense[a])
                    return fail(GBST_EINVAL, "source index outside the grid");
                const int64_t n = a == 0 ? s.lu.nx : a == 1 ? s.lu.ny : s.lu.nz;
                in = in && p[a] >= s.g0[a] && p[a] < s.g0[a] + n;
            }
            if (!in)
                continue;
            s.src_on = true;
            for (int a = 0; a < 3; ++a)
                s.src_local[a] = p[a] - s.g0[a];
            s.f0 = f0_hz;
            s.t0 = t0_s;
            s.amp = amp;
            GridDev &g = h->hgrids[i];
            g.has_src = 1;
            g.src_x = static_cast<int>(s.src_local[0]);
            g.src_y = static_cast<int>(s.src_local[1]);
            g.src_z = static_cast<int>(s.src_local[2]);
            placed = true;
        }
        if (!placed)
            return fail(GBST_EINVAL, "source index outside the grid");
    }
    GBST_CUDA(cudaMemcpyAsync(h->dgrids, h->hgrids.data(), h->hgrids.size() * sizeof(GridDev),
                              cudaMemcpyHostToDevice, h->stream));
    st = read_kappa_at_source(h);
    destroy_graphs(h);
    return st;
}

}  // namespace

// =========}  // namespace

// =========================================================================
extern "C" {

int gbst_version(void) { return 10000; }

const char *stencil_last_error(void) { return t_err.c_str(); }

gbst_status stencil_fd_weights(int space_order, double *out)
{
    if (!out || space_order < 2 || space_order > 16 || space_order % 2)
        return fail(GBST_EINVAL, "space_order must be even in [2, 16]");
    central_weights(space_order / 2, out);
    return GBST_OK;
}

gbst_status stencil_create(const gbst_desc *desc, gbst_handle *out)
{
    return create_handle(desc, 1, false, out);
}

gbst_status stencil_batch_create(const gbst_desc *descs, int n, gbst_handle *out)
{
    return create_handle(descs, n, true, out);
}

gbst_status stencil_system_create(const gbst_desc *desc, int nfields, const double *coupling, gbst_handle *out)
{
    if (!desc || !out || !coupling)
        return fail(GBST_EINVAL, "null argument");
    if (nfields < 2 || nfields > 4)
        return fail(GBST_EINVAL, "nfields must be 2, 3 or 4");
    for (int k = 0; k < nfields * nfields; ++k)
        if (!std::isfinite(coupling[k]))
            return fail(GBST_EINVAL, "coupling matrix entry %d is not finite", k);
    if (desc->eq != GBST_HEAT || desc->storage != GBST_F32 || desc->ndim != 3 || desc->bc != GBST_BC_ZERO ||
        desc->kernel == GBST_KERNEL_SIMPLE)
        return fail(GBST_ENOTSUP, "systems: heat-type, FP32, 3D, zero halos, streaming kernel");
    std::vector<gbst_desc> ds(nfields, *desc);
    for (auto &e : ds)
        e.temporal_block = 1;
    return create_handle(ds.data(), nfields, true, out, nfields, coupling);
}

gbst_status stencil_batch_size(gbst_handle h, int *n)
{
    if (!h || !n)
        return fail(GBST_EINVAL, "null argument");
    *n = h->members;
    return GBST_OK;
}

gbst_status stencil_destroy(gbst_handle h) { return destroy_handle(h); }

gbst_status stencil_set_field(gbst_handle h, int field, const void *src, int src_dtype, int src_on_device)
{
    return set_field_member(h, 0, field, src, src_dtype, src_on_device);
}

gbst_status stencil_batch_set_field(gbst_handle h, int grid, int field, const void *src, int src_dtype,
                                    int src_on_device)
{
    return set_field_member(h, grid, field, src, src_dtype, src_on_device);
}

gbst_status stencil_get_field(gbst_handle h, int field, void *dst, int dst_dtype, int dst_on_device)
{
    return transfer(h, 0, field, dst, dst_dtype, dst_on_device, false);
}

gbst_status stencil_batch_get_field(gbst_handle h, int grid, int field, void *dst, int dst_dtype, int dst_on_device)
{
    return transfer(h, grid, field, dst, dst_dtype, dst_on_device, false);
}

gbst_status stencil_set_field_async(gbst_handle h, int field, const void *src, int src_dtype, int src_on_device)
{
    return transfer(h, 0, field, const_cast<void *>(src), src_dtype, src_on_device, true, true);
}

gbst_status stencil_get_field_async(gbst_handle h, int field, void *dst, int dst_dtype, int dst_on_device)
{
    return transfer(h, 0, field, dst, dst_dtype, dst_on_device, false, true);
}

gbst_status stencil_set_source(gbst_handle h, const int64_t idx[3], double f0_hz, double t0_s, double amp)
{
    return set_source_member(h, 0, idx, f0_hz, t0_s, amp);
}

gbst_status stencil_batch_set_source(gbst_handle h, int grid, const int64_t idx[3], double f0_hz, double t0_s,
                                     double amp)
{
    return set_source_member(h, grid, idx, f0_hz, t0_s, amp);
}

gbst_status stencil_set_persistent(gbst_handle h, int enable)
{
    gbst_status st = check_handle(h);
    if (st != GBST_OK)
        return st;
    if (enable && h->closure)
        return fail(GBST_ENOTSUP, "persistent runs cannot apply a closure");
    if (enable && (!h->plan.stream || h->nboxes > 0))
        return fail(GBST_ENOTSUP, "persistent runs need the streaming kernel and no halo exchanges");
    h->persistent = enable != 0;
    destroy_graphs(h);
    return GBST_OK;
}

gbst_status stencil_attach_closure(gbst_handle h, gbst_closure c, double c_ref)
{
    gbst_status st = check_handle(h);
    if (st != GBST_OK)
        return st;
    destroy_graphs(h);
    if (!c) {
        h->closure = nullptr;
        return GBST_OK;
    }
    if (h->d.eq != GBST_WAVE || h->ndim != 3 || h->subs.size() != 1)
        return fail(GBST_ENOTSUP, "closures apply to a single undecomposed 3D wave grid");
    if (h->persistent)
        return fail(GBST_ENOTSUP, "closures cannot run in persistent mode");
    if (!(c_ref > 0.0))
        return fail(GBST_EINVAL, "c_ref must be positive");
    const Sub &sb = h->subs[0];
    const int64_t n = sb.lu.nx * sb.lu.ny * sb.lu.nz;
    if (!h->cl_up) {
        h->cl_up = static_cast<float *>(dalloc(h, n * sizeof(float)));
        h->cl_un = static_cast<float *>(dalloc(h, n * sizeof(float)));
        h->cl_cn = static_cast<float *>(dalloc(h, n * sizeof(float)));
        h->cl_corr = static_cast<float *>(dalloc(h, n * sizeof(float)));
        if (!h->cl_up || !h->cl_un || !h->cl_cn || !h->cl_corr)
            return fail(GBST_ENOMEM, "closure work buffers");
    }
    XferArgs x{};
    x.padded = h->hgrids[0].kappa;
    x.storage = GBST_F32;
    x.pitch = sb.lk.pitch;
    x.rows = sb.lk.rows;
    x.origin = sb.lk.origin;
    x.nx = sb.lk.nx;
    x.ny = sb.lk.ny;
    x.nz = sb.lk.nz;
    x.dense = h->cl_cn;
    GBST_CUDA(launch_kappa_to_cnorm(x, sb.h / (sb.dt * c_ref), h->stream));
    if (closure_stream(c) != h->stream)
        return fail(GBST_EINVAL, "the closure and the grid must use the same stream");
    h->closure = c;
    GBST_CUDA(cudaStreamSynchronize(h->stream));
    return GBST_OK;
}

// Gradient of a rollout loss of the attached closure, by backpropagation through the
// coarse time steps (see gbstencil.h).
gbst_status stencil_closure_rollout_grad(gbst_handle h, const float *u_cur, const float *u_prev, int64_t step0,
                                         const float *const *refs, int nsteps, double *loss)
{
    gbst_status st = check_handle(h);
    if (st != GBST_OK)
        return st;
    if (!u_cur || !u_prev || !refs || !loss || nsteps < 1 || nsteps > 4096)
        return fail(GBST_EINVAL, "stencil_closure_rollout_grad: null argument or nsteps not in [1, 4096]");
    for (int j = 0; j < nsteps; ++j)
        if (!refs[j])
            return fail(GBST_EINVAL, "stencil_closure_rollout_grad: refs[%d] is null", j);
    gbst_closure c = h->closure;
    if (!c || !closure_has_features(c))
        return fail(GBST_ENOTSUP, "stencil_closure_rollout_grad: needs an attached closure with feature inputs");
    const Sub &sb = h->subs[0];
    const int64_t nx = sb.lu.nx, ny = sb.lu.ny, nz = sb.lu.nz, n = nx * ny * nz;
    const size_t fb = static_cast<size_t>(n) * sizeof(float);
    cudaStream_t s = h->stream;
    // work buffers, kept for later calls
    if (h->roll_cap < nsteps) {
        while (static_cast<int>(h->roll_up.size()) < nsteps) {
            float *a = static_cast<float *>(dalloc(h, fb)), *b = static_cast<float *>(dalloc(h, fb)),
                  *c2 = static_cast<float *>(dalloc(h, fb));
            if (!a || !b || !c2)
                return fail(GBST_ENOMEM, "rollout buffers (%d steps of %lld points)", nsteps,
                            static_cast<long long>(n));
            h->roll_up.push_back(a);
            h->roll_un.push_back(b);
            h->roll_u.push_back(c2);
        }
        if (!h->roll_A) {
            for (auto &pa : h->roll_a)
                pa = static_cast<float *>(dalloc(h, fb));
            h->roll_A = static_cast<float *>(dalloc(h, fb));
            h->roll_gun = static_cast<float *>(dalloc(h, fb));
            h->roll_kap = static_cast<float *>(dalloc(h, fb));
            if (!h->roll_a[0] || !h->roll_a[1] || !h->roll_a[2] || !h->roll_A || !h->roll_gun || !h->roll_kap)
                return fail(GBST_ENOMEM, "rollout buffers");
        }
        h->roll_sums = static_cast<double *>(dalloc(h, 2 * sizeof(double) * static_cast<size_t>(nsteps)));
        if (!h->roll_sums)
            return fail(GBST_ENOMEM, "rollout buffers");
        h->roll_cap = nsteps;
    }
    // dense kappa of the grid (the leapfrog step's coefficient)
    XferArgs xk{};
    xk.padded = h->hgrids[0].kappa;
    xk.storage = GBST_F32;
    xk.pitch = sb.lk.pitch;
    xk.rows = sb.lk.rows;
    xk.origin = sb.lk.origin;
    xk.nx = nx;
    xk.ny = ny;
    xk.nz = nz;
    xk.gnx = nx;
    xk.gny = ny;
    xk.dense_dtype = GBST_F32;
    xk.dense = h->roll_kap;
    GBST_CUDA(launch_gather(xk, s));
    // forward: nsteps corrected steps from (u_cur, u_prev), keeping u+, u^n and u^{n+1}
    if ((st = stencil_set_field(h, GBST_U, u_cur, GBST_F32, 1)) != GBST_OK ||
        (st = stencil_set_field(h, GBST_U_PREV, u_prev, GBST_F32, 1)) != GBST_OK ||
        (st = stencil_set_step(h, step0)) != GBST_OK)
        return st;
    XferArgs xu = xk;
    xu.storage = h->d.storage;
    xu.pitch = sb.lu.pitch;
    xu.rows = sb.lu.rows;
    xu.origin = sb.lu.origin;
    for (int j = 0; j < nsteps; ++j) {
        if ((st = stencil_run(h, 1)) != GBST_OK)
            return st;
        GBST_CUDA(cudaMemcpyAsync(h->roll_up[j], h->cl_up, fb, cudaMemcpyDeviceToDevice, s));
        GBST_CUDA(cudaMemcpyAsync(h->roll_un[j], h->cl_un, fb, cudaMemcpyDeviceToDevice, s));
        xu.padded = h->hgrids[0].buf[h->parity];
        xu.dense = h->roll_u[j];
        GBST_CUDA(launch_gather(xu, s));
    }
    // loss = mean over the steps of |u^{n0+j+1} - ref_j|^2 / |ref_j|^2; roll_u[j] <- its gradient
    GBST_CUDA(cudaMemsetAsync(h->roll_sums, 0, 2 * sizeof(double) * static_cast<size_t>(nsteps), s));
    for (int j = 0; j < nsteps; ++j) {
        if ((st = rollout_sums(h->roll_u[j], refs[j], n, h->roll_sums + 2 * j, s)) != GBST_OK ||
            (st = rollout_grad(h->roll_u[j], refs[j], n, h->roll_sums + 2 * j, 1.0 / nsteps, s)) != GBST_OK)
            return st;
    }
    // backward: a_next = cotangent of u^{n0+j+1}, a_cur of u^{n0+j}, a_prev of u^{n0+j-1}
    float *a_next = h->roll_a[0], *a_cur = h->roll_a[1], *a_prev = h->roll_a[2];
    GBST_CUDA(cudaMemcpyAsync(a_next, h->roll_u[nsteps - 1], fb, cudaMemcpyDeviceToDevice, s));
    if (nsteps >= 2)
        GBST_CUDA(cudaMemcpyAsync(a_cur, h->roll_u[nsteps - 2], fb, cudaMemcpyDeviceToDevice, s));
    for (int j = nsteps - 1; j >= 0; --j) {
        st = closure_backward(c, h->roll_up[j], h->roll_un[j], h->cl_cn, nx, ny, nz, a_next, h->roll_A, h->roll_gun,
                              j < nsteps - 1 ? 1 : 0);
        if (st != GBST_OK)
            return st;
        if (j == 0)
            break;  // the initial levels are given, their cotangents are not needed
        // u+ = 2 u^n - u^{n-1} + kappa L u^n (+ source): a_cur += 2A + L(kappa A) + gun, a_prev = -A (+ loss)
        st = stencil_wave_adjoint_dense(h->d.space_order, nx, ny, nz, h->roll_kap, h->roll_A, a_cur, a_prev, s);
        if (st != GBST_OK)
            return st;
        if ((st = dense_axpy(a_cur, h->roll_gun, 1.0f, n, s)) != GBST_OK)
            return st;
        if (j >= 2 && (st = dense_axpy(a_prev, h->roll_u[j - 2], 1.0f, n, s)) != GBST_OK)
            return st;
        float *t = a_next;
        a_next = a_cur;
        a_cur = a_prev;
        a_prev = t;
    }
    std::vector<double> sums(2 * static_cast<size_t>(nsteps));
    GBST_CUDA(cudaMemcpyAsync(sums.data(), h->roll_sums, sums.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
    GBST_CUDA(cudaStreamSynchronize(s));
    double l = 0.0;
    for (int j = 0; j < nsteps; ++j)
        l += sums[2 * j + 1] > 0.0 ? sums[2 * j] / sums[2 * j + 1] : 0.0;
    *loss = l / nsteps;
    return poll_device_error(h);
}

gbst_status stencil_get_field_strided(gbst_handle h, int field, float *dst, int stride)
{
    gbst_status st = check_handle(h);
    if (st != GBST_OK)
        return st;
    if (!dst || stride < 1)
        return fail(GBST_EINVAL, "null destination or stride < 1");
    if (h->subs.size() != 1)
        return fail(GBST_ENOTSUP, "strided reads need a single undecomposed grid");
    if (field != GBST_U && field != GBST_U_PREV)
        return fail(GBST_EINVAL, "strided reads support GBST_U and GBST_U_PREV");
    if (h->d.eq == GBST_HEAT && field != GBST_U)
        return fail(GBST_EINVAL, "heat grids have only the field GBST_U");
    const Sub &sb = h->subs[0];
    XferArgs x{};
    x.padded = h->hgrids[0].buf[field == GBST_U ? h->parity : 1 - h->parity];
    x.storage = h->d.storage;
    x.pitch = sb.lu.pitch;
    x.rows = sb.lu.rows;
    x.origin = sb.lu.origin;
    x.nx = sb.lu.nx;
    x.ny = sb.lu.ny;
    x.nz = sb.lu.nz;
    x.dense = dst;
    GBST_CUDA(launch_gather_strided(x, stride, h->stream));
    return poll_device_error(h);
}

gbst_status stencil_debug_barrier_extra(gbst_handle h, unsigned int extra)
{
    if (!h)
        return fail(GBST_EINVAL, "null handle");
    h->barrier_extra = extra;
    destroy_graphs(h);
    return GBST_OK;
}

gbst_status stencil_run(gbst_handle h, int64_t nsteps)
{
    gbst_status st = check_handle(h);
    if (st != GBST_OK)
        return st;
    if (nsteps < 0)
        return fail(GBST_EINVAL, "nsteps must be >= 0");
    if (nsteps == 0)
        return GBST_OK;
    if (nsteps > (int64_t(1) << 30))
        return fail(GBST_EINVAL, "nsteps too large for one call");
    for (const Sub &s : h->subs)
        if (s.unstable && !h->d.allow_unstable)
            return fail(GBST_EUNSTABLE, "velocity model exceeds the stability limit");
    const int64_t ns = static_cast<int64_t>(h->subs.size());
    bool src = false;
    for (const Sub &s : h->subs)
        src = src || (h->d.eq == GBST_WAVE && s.src_on);
    if (src) {
        st = ensure_src_capacity(h, nsteps);
        if (st != GBST_OK)
            return st;
        if (h->src_ev)
            GBST_CUDA(cudaEventSynchronize(h->src_ev));  // previous upload finished reading hsrc
        else
            GBST_CUDA(cudaEventCreateWithFlags(&h->src_ev, cudaEventDisableTiming));
        for (int64_t i = 0; i < ns; ++i) {
            const Sub &s = h->subs[i];
            const double scale = s.src_on ? s.amp * s.kappa_src * s.h * s.h : 0.0;
            for (int64_t k = 0; k < nsteps; ++k)
                h->hsrc[k * ns + i] =
                    s.src_on ? static_cast<float>(scale * ricker((h->step + k) * s.dt, s.f0, s.t0)) : 0.f;
        }
        GBST_CUDA(cudaMemcpyAsync(h->dsrc, h->hsrc, nsteps * ns * sizeof(float), cudaMemcpyHostToDevice, h->stream));
        GBST_CUDA(cudaEventRecord(h->src_ev, h->stream));
    }
    const bool tb = h->plan.stream && h->plan.var.tb == 2;
    const bool persistent = h->persistent && h->plan.stream && h->nboxes == 0 && !tb && h->nf == 1;
    // sweep launches: one per step, or one per two steps (+ one single step if odd)
    const int64_t launches = persistent ? 1 : (tb ? (nsteps + 1) / 2 : nsteps);
    if (h->profile) {
        const int64_t need = 2 * launches;
        while (static_cast<int64_t>(h->prof_ev.size()) < need) {
            cudaEvent_t e;
            GBST_CUDA(cudaEventCreate(&e));
            h->prof_ev.push_back(e);
        }
        h->prof_launches = launches;
    }
    auto enqueue_all = [&]() -> gbst_status {
        if (persistent)
            return enqueue_persistent(h, nsteps, h->parity, src ? h->dsrc : nullptr, h->profile);
        int par = h->parity;
        for (int64_t k = 0; k < launches; ++k) {
            const bool single = tb && 2 * k + 1 == nsteps;
            gbst_status s2 = enqueue_step(h, par, src ? h->dsrc + k * ns : nullptr,
                                          h->profile ? static_cast<int>(k) : -1, single);
            if (s2 != GBST_OK)
                return s2;
            par ^= 1;
        }
        return GBST_OK;
    };
    // (a closure's weights may change between runs: its steps are launched directly)
    const bool graph = h->d.use_graph && h->stream != nullptr && !h->closure;
    if (graph) {
        const auto key = std::make_pair(nsteps, h->parity + (h->profile ? 2 : 0) + (persistent ? 4 : 0));
        auto it = h->graphs.find(key);
        if (it == h->graphs.end()) {
            GBST_CUDA(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
            st = enqueue_all();
            cudaGraph_t g = nullptr;
            const cudaError_t ec = cudaStreamEndCapture(h->stream, &g);
            if (st != GBST_OK) {
                if (g)
                    cudaGraphDestroy(g);
                return st;
            }
            if (ec != cudaSuccess)
                return fail(GBST_ECUDA, "graph capture: %s", cudaGetErrorString(ec));
            cudaGraphExec_t ge = nullptr;
            cudaError_t e = cudaGraphInstantiate(&ge, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess)
                return fail(GBST_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
            it = h->graphs.emplace(key, ge).first;
        }
        GBST_CUDA(cudaGraphLaunch(it->second, h->stream));
    } else {
        st = enqueue_all();
        if (st != GBST_OK)
            return st;
    }
    h->parity ^= static_cast<int>((persistent ? nsteps : launches) & 1);
    h->step += nsteps;
    return GBST_OK;
}

gbst_status stencil_sync(gbst_handle h)
{
    gbst_status st = check_handle(h);
    if (st != GBST_OK)
        return st;
    return poll_device_error(h);
}

gbst_status stencil_get_step(gbst_handle h, int64_t *step)
{
    if (!h || !step)
        return fail(GBST_EINVAL, "null argument");
    *step = h->step;
    return GBST_OK;
}

gbst_status stencil_set_step(gbst_handle h, int64_t step)
{
    if (!h || step < 0)
        return fail(GBST_EINVAL, "bad argument");
    h->step = step;
    return GBST_OK;
}

static gbst_status reduce_api(gbst_handle h, int member, int kind, double *out)
{
    gbst_status st = check_handle(h);
    if (st != GBST_OK)
        return st;
    if (!out)
        return fail(GBST_EINVAL, "null out");
    if (kind < GBST_RED_SUM || kind > GBST_RED_ENERGY)
        return fail(GBST_EINVAL, "unknown reduction %d", kind);
    if (member >= h->members)
        return fail(GBST_EINVAL, "grid index %d out of range", member);
    if (kind == GBST_RED_ENERGY && h->d.eq != GBST_WAVE)
        return fail(GBST_EINVAL, "the energy reduction is defined for the wave equation only");
    if (kind == GBST_RED_ENERGY && h->nboxes > 0) {
        // ghosts of u^{n-1}: swap / wrap them so the stencil in the energy sees neighbours
        cudaError_t e = launch_halo_copies(h->dgrids, h->dboxes, h->nboxes, 1 - h->parity, h->es, h->copy_blocks,
                                           h->stream);
        if (e != cudaSuccess)
            return fail(GBST_ECUDA, "halo copies: %s", cudaGetErrorString(e));
    }
    double v = 0.0;
    st = reduce_member(h, member, kind, 0, &v);
    if (st != GBST_OK)
        return st;
    *out = v;
    if (!std::isfinite(v))
        return fail(GBST_EUNSTABLE, "reduction result is not finite");
    return GBST_OK;
}

gbst_status stencil_reduce_f64(gbst_handle h, int kind, double *out) { return reduce_api(h, -1, kind, out); }

gbst_status stencil_batch_reduce_f64(gbst_handle h, int grid, int kind, double *out)
{
    return reduce_api(h, grid, kind, out);
}

gbst_status stencil_describe(gbst_handle h, char *buf, size_t len)
{
    if (!h || !buf || len == 0)
        return fail(GBST_EINVAL, "bad argument");
    const Plan &p = h->plan;
    const int px = px_of(h->d.storage);
    snprintf(buf, len,
             "{\"kernel\": \"%s\", \"R\": %d, \"threads\": %d, \"py\": %d, \"depth\": %d, \"tile\": [%d, %d], "
             "\"zchunks\": %d, \"units\": %d, \"ctas\": %d, \"occupancy\": %d, \"smem\": %zu, \"subdomains\": %zu, "
             "\"halo_boxes\": %d, \"variant\": %d, \"minb\": %d, \"tb\": %d, \"ys\": %d, \"nf\": %d, \"dyn\": %d, "
             "\"overlap\": %d, \"interior_units\": %d, \"opt\": %d}",
             p.stream ? "stream" : "simple", h->R, p.var.nthreads, p.var.py, p.var.depth, tile_w(p.var, px),
             p.stream ? tile_h(p.var) : (p.var.nthreads / std::max(1, p.txt)) * p.var.py, p.zchunks, p.nunits,
             p.ctas, p.occupancy, p.smem, h->subs.size(), h->nboxes, p.variant, p.var.minb,
             p.stream ? p.var.tb : 1, p.stream && p.var.ys ? 1 : 0, h->nf, p.dyn ? 1 : 0, p.overlap ? 1 : 0,
             p.nint, p.stream ? p.var.opt : 0);
    return GBST_OK;
}

gbst_status stencil_set_profile(gbst_handle h, int enable)
{
    if (!h)
        return fail(GBST_EINVAL, "null handle");
    h->profile = enable != 0;
    return GBST_OK;
}

gbst_status stencil_last_kernel_time(gbst_handle h, double *ms, int64_t *launches)
{
    gbst_status st = check_handle(h);
    if (st != GBST_OK)
        return st;
    if (!ms || !launches)
        return fail(GBST_EINVAL, "null argument");
    st = poll_device_error(h);
    if (st != GBST_OK)
        return st;
    double tot = 0.0;
    for (int64_t k = 0; k < h->prof_launches; ++k) {
        float t = 0.f;
        GBST_CUDA(cudaEventElapsedTime(&t, h->prof_ev[2 * k], h->prof_ev[2 * k + 1]));
        tot += t;
    }
    *ms = tot;
    *launches = h->prof_launches;
    return GBST_OK;
}

gbst_status stencil_set_plan(gbst_handle h, int variant, int txt, int zchunks, int ctas)
{
    gbst_status st = check_handle(h);
    if (st != GBST_OK)
        return st;
    GBST_CUDA(cudaStreamSynchronize(h->stream));
    return build_plan(h, variant, txt, zchunks, ctas);
}

gbst_status stencil_set_schedule(gbst_handle h, int dynamic)
{
    gbst_status st = check_handle(h);
    if (st != GBST_OK)
        return st;
    if (dynamic < -1 || dynamic > 1)
        return fail(GBST_EINVAL, "schedule must be -1 (default), 0 (static) or 1 (dynamic)");
    GBST_CUDA(cudaStreamSynchronize(h->stream));
    h->dyn_pref = dynamic;
    return build_plan(h, h->plan.variant, h->plan.req_txt, h->plan.req_zchunks, h->plan.req_ctas);
}

gbst_status stencil_set_overlap(gbst_handle h, int enable)
{
    gbst_status st = check_handle(h);
    if (st != GBST_OK)
        return st;
    if (enable < -1 || enable > 1)
        return fail(GBST_EINVAL, "overlap must be -1 (default), 0 (off) or 1 (on)");
    GBST_CUDA(cudaStreamSynchronize(h->stream));
    h->overlap_pref = enable;
    return build_plan(h, h->plan.variant, h->plan.req_txt, h->plan.req_zchunks, h->plan.req_ctas);
}

int stencil_variant_count(void) { return stream_variant_count(); }

gbst_status stencil_variant_info(int i, char *buf, size_t len)
{
    StreamVariant v;
    if (!buf || len == 0 || !stream_variant_get(i, &v))
        return fail(GBST_EINVAL, "bad variant index or buffer");
    snprintf(buf, len,
             "{\"R\": %d, \"eq\": %d, \"storage\": %d, \"has_z\": %d, \"threads\": %d, \"py\": %d, \"depth\": %d, "
             "\"minb\": %d, \"txt\": %d, \"tb\": %d, \"ys\": %d, \"nf\": %d, \"opt\": %d}",
             v.R, v.eq, v.storage, v.has_z ? 1 : 0, v.nthreads, v.py, v.depth, v.minb, v.txt, v.tb, v.ys ? 1 : 0,
             v.nf, v.opt);
    return GBST_OK;
}

gbst_status stencil_tune(gbst_handle h, int reps, char *report, size_t len)
{
    gbst_status st = check_handle(h);
    if (st != GBST_OK)
        return st;
    if (!h->plan.stream) {
        if (report && len)
            snprintf(report, len, "{\"tuned\": false, \"reason\": \"simple kernel\"}");
        return GBST_OK;
    }
    reps = std::max(1, reps);
    GBST_CUDA(cudaStreamSynchronize(h->stream));
    // Repeated launches at a fixed parity leave u^n intact; the wave's in-place
    // update overwrites u^{n-1}, so that buffer is saved and restored.
    std::vector<void *> saved(h->subs.size(), nullptr);
    auto restore = [&]() {
        for (size_t i = 0; i < h->subs.size(); ++i)
            if (saved[i]) {
                cudaMemcpyAsync(h->hgrids[i].buf[1 - h->parity], saved[i], h->subs[i].lu.bytes,
                                cudaMemcpyDeviceToDevice, h->stream);
                cudaStreamSynchronize(h->stream);
                h->mem.release(saved[i], h->subs[i].lu.bytes);
                saved[i] = nullptr;
            }
    };
    if (h->d.eq == GBST_WAVE)
        for (size_t i = 0; i < h->subs.size(); ++i) {
            saved[i] = h->mem.alloc(h->subs[i].lu.bytes);
            if (!saved[i]) {
                restore();
                return fail(GBST_ENOMEM, "autotuner save buffer");
            }
            GBST_CUDA(cudaMemcpyAsync(saved[i], h->hgrids[i].buf[1 - h->parity], h->subs[i].lu.bytes,
                                      cudaMemcpyDeviceToDevice, h->stream));
        }
    cudaEvent_t e0, e1;
    GBST_CUDA(cudaEventCreate(&e0));
    GBST_CUDA(cudaEventCreate(&e1));
    const Plan before = h->plan;
    double best_ms = 1e300;
    const int pref_before = h->dyn_pref;
    const bool overlap_wanted =
        h->nboxes > 0 && (h->overlap_pref == 1 || (h->overlap_pref < 0 && kOverlapDefault));
    TunedPlan best{before.variant, before.req_txt, before.req_zchunks, before.req_ctas, pref_before};
    std::string rep = "{\"candidates\": [";
    int ncand = 0;
    StreamVariant v;
    const int zlist_3d[] = {0, 1, 2, 4, 8, 16};
    const int zlist_2d[] = {0};
    for (int vi = 0; stream_variant_get(vi, &v); ++vi) {
        if (!variant_matches(h, v))
            continue;
        {
            const int txt = v.txt;
            const bool chunked = h->ndim == 3 || v.ys;
            const int *zl = chunked ? zlist_3d : zlist_2d;
            const int nz = chunked ? 6 : 1;
            int last_units = -1;
            // static and dynamic unit assignment
            const int ndyn = 2;
            for (int zi = 0; zi < nz * ndyn; ++zi) {
                const int dv = zi % ndyn;
                h->dyn_pref = dv;
                if (build_plan(h, vi, txt, zl[zi / ndyn], 0) != GBST_OK)
                    continue;
                if (dv == 0 && h->plan.nunits == last_units) {
                    zi += ndyn - 1;  // same units as the previous z-chunking: skip it
                    continue;
                }
                last_units = h->plan.nunits;
                // with the halo-exchange overlap requested, only plans that can split
                // (the tuner times sweeps without copies and cannot weigh the overlap)
                if (overlap_wanted && !h->plan.overlap)
                    continue;
                const SweepArgs a = sweep_args(h, h->parity, nullptr);
                cudaError_t e = launch_stream_sweep(h->plan.var, a, h->plan.ctas, h->plan.smem, h->stream);
                cudaEventRecord(e0, h->stream);
                for (int r = 0; r < reps && e == cudaSuccess; ++r)
                    e = launch_stream_sweep(h->plan.var, a, h->plan.ctas, h->plan.smem, h->stream);
                cudaEventRecord(e1, h->stream);
                if (e != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
                    cudaGetLastError();
                    continue;
                }
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                const double per = ms / reps / v.tb;  // per time step
                char b[256];
                snprintf(b, sizeof b,
                         "%s{\"variant\": %d, \"txt\": %d, \"zchunks\": %d, \"units\": %d, \"ctas\": %d, "
                         "\"tb\": %d, \"dyn\": %d, \"ms\": %.5f}",
                         ncand ? ", " : "", vi, txt, h->plan.zchunks, h->plan.nunits, h->plan.ctas, v.tb,
                         h->plan.dyn ? 1 : 0, per);
                rep += b;
                ++ncand;
                if (per < best_ms) {
                    best_ms = per;
                    best = TunedPlan{vi, txt, h->plan.zchunks, 0, h->plan.dyn ? 1 : 0};
                }
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    h->dyn_pref = best.dyn;
    st = build_plan(h, best.variant, best.txt, best.zchunks, best.ctas);
    restore();
    gbst_status pe = poll_device_error(h);
    if (st != GBST_OK)
        return st;
    if (pe != GBST_OK)
        return pe;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        tune_cache_load();
        tune_cache_store(tune_key(h), best);
    }
    char b[256];
    snprintf(b, sizeof b, "], \"best\": {\"variant\": %d, \"txt\": %d, \"zchunks\": %d, \"dyn\": %d, \"ms\": %.5f}}",
             best.variant, best.txt, best.zchunks, h->plan.dyn ? 1 : 0, best_ms);
    rep += b;
    if (report && len) {
        strncpy(report, rep.c_str(), len - 1);
        report[len - 1] = 0;
    }
    return GBST_OK;
}

}  // extern "C"

