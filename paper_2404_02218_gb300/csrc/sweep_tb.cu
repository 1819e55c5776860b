// Temporally blocked heat variants (two steps per launch, FP32, 3D): radius,
// main warps, rows per thread, prefetch depth, min blocks.  The tile height is
// main warps x rows per thread - 2r.  Radius 4 is not blocked: its two queues
// do not fit the register file without spilling.
#include "sweep_tb.cuh"

namespace gbst {
namespace sweep {
namespace {
const Entry kTable[] = {
    tb_entry<1, 9, 2, 2, 1>(),
    tb_entry<1, 8, 2, 2, 1>(),
    tb_entry<1, 16, 1, 2, 1>(),
    tb_entry<1, 10, 1, 3, 1>(),
    tb_entry<1, 12, 2, 2, 1>(),
    tb_entry<1, 8, 2, 2, 2>(),
    tb_entry<1, 10, 1, 2, 2>(),
    tb_entry<1, 6, 2, 2, 2>(),
    tb_entry<2, 10, 2, 2, 1>(),
    tb_entry<2, 12, 1, 2, 1>(),
    tb_entry<2, 16, 1, 2, 1>(),
};
}  // namespace

const Entry *table_tb(int *n)
{
    *n = static_cast<int>(sizeof(kTable) / sizeof(kTable[0]));
    return kTable;
}
}  // namespace sweep
}  // namespace gbst
