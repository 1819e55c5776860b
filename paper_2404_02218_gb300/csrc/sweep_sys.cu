// Fused multi-field system variants (FP32, 3D): radius, fields, consumer
// warps, rows per thread, prefetch depth, min blocks, tile threads in x.
#include "sweep_sys.cuh"

namespace gbst {
namespace sweep {
namespace {
const Entry kTable[] = {
    sys_entry<1, 3, 4, 1, 3, 2, 32>(),
    sys_entry<1, 3, 4, 2, 3, 1, 32>(),
    sys_entry<2, 3, 4, 1, 3, 2, 32>(),
    sys_entry<2, 3, 4, 1, 2, 2, 32>(),
    sys_entry<4, 3, 4, 1, 3, 1, 32>(),
    sys_entry<1, 2, 4, 2, 3, 2, 32>(),
    sys_entry<2, 2, 4, 1, 3, 2, 32>(),
    sys_entry<4, 2, 4, 1, 3, 1, 32>(),
    sys_entry<1, 4, 4, 1, 3, 2, 32>(),
    sys_entry<2, 4, 4, 1, 2, 1, 32>(),
    sys_entry<4, 4, 4, 1, 2, 1, 32>(),
};
}  // namespace

const Entry *table_sys(int *n)
{
    *n = static_cast<int>(sizeof(kTable) / sizeof(kTable[0]));
    return kTable;
}
}  // namespace sweep
}  // namespace gbst
