// Temporally blocked heat variants (two steps per launch, FP32, 3D): radius,
// main warps, rows per thread, prefetch depth, min blocks.  The tile height is
// main warps x rows per thread - 2r.  Three or four rows per thread spread the
// per-iteration work (barriers, addresses, queue handling) over more points and
// measured 14 % faster than two at order 2; radius 2 keeps two rows (its two
// 5-plane queues leave no registers for more).  Radius 4 is not blocked: its
// two queues do not fit the register file without spilling.
#include "sweep_tb.cuh"

namespace gbst {
namespace sweep {
namespace {
const Entry kTable[] = {
    tb_entry<1, 10, 3, 3, 1>(),
    tb_entry<1, 10, 3, 2, 1>(),
    tb_entry<1, 9, 3, 2, 1>(),
    tb_entry<1, 10, 4, 2, 1>(),
    tb_entry<1, 9, 4, 2, 1>(),
    tb_entry<1, 8, 4, 2, 1>(),
    tb_entry<1, 12, 2, 2, 1>(),
    tb_entry<1, 6, 2, 2, 2>(),
    tb_entry<2, 10, 2, 2, 1>(),
};
}  // namespace

const Entry *table_tb(int *n)
{
    *n = static_cast<int>(sizeof(kTable) / sizeof(kTable[0]));
    return kTable;
}
}  // namespace sweep
}  // namespace gbst
