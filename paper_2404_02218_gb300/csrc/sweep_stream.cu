// Registry of the streaming-sweep variants compiled in sweep_r*.cu, and the
// host-side launch helpers.
#include "sweep_stream.cuh"

namespace gbst {
namespace sweep {
const Entry *table_r1(int *n);
const Entry *table_r2(int *n);
const Entry *table_r4(int *n);
const Entry *table_tb(int *n);
const Entry *table_r1_2d(int *n);
const Entry *table_r2_2d(int *n);
const Entry *table_r4_2d(int *n);
const Entry *table_sys(int *n);
const Entry *table_r2_rows4(int *n);
const Entry *table_sx(int *n);
}  // namespace sweep

namespace {
using sweep::Entry;

struct Registry {
    static constexpr int kTables = 10;
    const Entry *tab[kTables];
    int n[kTables];
    Registry()
    {
        tab[0] = sweep::table_r1(&n[0]);
        tab[1] = sweep::table_r2(&n[1]);
        tab[2] = sweep::table_r4(&n[2]);
        tab[3] = sweep::table_tb(&n[3]);
        tab[4] = sweep::table_r1_2d(&n[4]);
        tab[5] = sweep::table_r2_2d(&n[5]);
        tab[6] = sweep::table_r4_2d(&n[6]);
        tab[7] = sweep::table_sys(&n[7]);
        tab[8] = sweep::table_r2_rows4(&n[8]);
        tab[9] = sweep::table_sx(&n[9]);
    }
    int total() const
    {
        int t = 0;
        for (int i = 0; i < kTables; ++i)
            t += n[i];
        return t;
    }
    const Entry *at(int i) const
    {
        for (int t = 0; t < kTables; ++t) {
            if (i < n[t])
                return &tab[t][i];
            i -= n[t];
        }
        return nullptr;
    }
};

const Registry &registry()
{
    static const Registry r;
    return r;
}

const Entry *find(const StreamVariant &v)
{
    const Registry &r = registry();
    for (int i = 0; i < r.total(); ++i) {
        const Entry *e = r.at(i);
        if (e->v.R == v.R && e->v.eq == v.eq && e->v.storage == v.storage && e->v.has_z == v.has_z &&
            e->v.nthreads == v.nthreads && e->v.py == v.py && e->v.depth == v.depth && e->v.minb == v.minb &&
            e->v.txt == v.txt && e->v.tb == v.tb && e->v.ys == v.ys && e->v.nf == v.nf && e->v.opt == v.opt)
            return e;
    }
    return nullptr;
}

// Allow the kernel the device's whole opt-in shared memory once, so handles with
// different slot sizes can share the function.
bool allow_max_smem(const Entry *e)
{
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
        return false;
    return cudaFuncSetAttribute(reinterpret_cast<const void *>(e->fn), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                optin) == cudaSuccess;
}

}  // namespace

bool stream_variant_exists(const StreamVariant &v) { return find(v) != nullptr; }

int stream_variant_count() { return registry().total(); }

bool stream_variant_get(int i, StreamVariant *v)
{
    const Entry *e = registry().at(i);
    if (i < 0 || !e)
        return false;
    *v = e->v;
    return true;
}

// Shared memory beyond the barrier header and the plane ring.  Wave: per
// barrier pair, kappa (FP32) and u^{n-1} of the centre plane (tile only).
// Temporally blocked heat: r + 2 step-1 planes of the grown tile plus r rows of
// slack (rows a main warp may read past the last plane, results discarded).
static size_t centre_bytes(const StreamVariant &v)
{
    if (v.tb == 2) {
        const size_t uw = static_cast<size_t>(tile_w(v, 4)) + 8, uh = static_cast<size_t>(tile_h(v)) + 2 * v.R;
        const size_t plane = (uw * uh * 4 + 127) / 128 * 128;
        const size_t pad = (static_cast<size_t>(v.R) * uw * 4 + 127) / 128 * 128;
        return plane * (v.R + 2) + pad;
    }
    if (v.eq != GBST_WAVE)
        return 0;
    const int px = px_of(v.storage), es = v.storage == GBST_BF16 ? 2 : 4;
    const size_t tx = static_cast<size_t>(v.txt) * px, ty = static_cast<size_t>(v.nthreads / v.txt) * v.py;
    const size_t slot = (tx * ty * (4 + es) + 127) / 128 * 128;
    return slot * (v.depth + 1);
}

size_t stream_smem_bytes(const StreamVariant &v, int max_box_bytes)
{
    const int rz = stream_rz(v);
    const int slots = (rz + 1 + v.depth) * v.nf;  // a multi-field sweep holds nf boxes per plane
    const size_t slot = (static_cast<size_t>(max_box_bytes) + 127) / 128 * 128;
    return 256 + slots * slot + centre_bytes(v);
}

int stream_slot_bytes(const StreamVariant &v, size_t smem)
{
    const int rz = stream_rz(v);
    const int slots = (rz + 1 + v.depth) * v.nf;
    return static_cast<int>((smem - 256 - centre_bytes(v)) / slots);
}

int stream_occupancy(const StreamVariant &v, size_t smem)
{
    const Entry *e = find(v);
    if (!e || !allow_max_smem(e))
        return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, e->fn, block_threads(v), smem) != cudaSuccess)
        return 0;
    return n;
}

cudaError_t launch_stream_sweep(const StreamVariant &v, const SweepArgs &a, int ctas, size_t smem, cudaStream_t s,
                                bool cooperative)
{
    const Entry *e = find(v);
    if (!e)
        return cudaErrorInvalidDeviceFunction;
    const int slot_bytes = stream_slot_bytes(v, smem);
    if (!cooperative) {
        e->fn<<<ctas, block_threads(v), smem, s>>>(a, slot_bytes);
        return cudaGetLastError();
    }
    // persistent launch: every CTA must be resident for the grid barrier
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(ctas);
    cfg.blockDim = dim3(block_threads(v));
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, e->fn, a, slot_bytes);
}

}  // namespace gbst
