// Streaming-sweep variants of radius 2 (space order 4), 3D grids.  The first
// entry matching a grid's (equation, storage) is its default.
#include "sweep_stream.cuh"

namespace gbst {
namespace sweep {
namespace {
const Entry kTable[] = {
    GBST_EQS(2, GBST_F32, true, 4, 2, 3, 1, 32),
    GBST_EQS(2, GBST_F32, true, 4, 1, 3, 4, 32),
    GBST_EQS(2, GBST_F32, true, 4, 2, 5, 2, 32),
    GBST_EQS(2, GBST_F32, true, 4, 2, 7, 2, 32),
    GBST_EQS(2, GBST_F32, true, 4, 2, 5, 2, 16),
    GBST_EQS(2, GBST_F32, true, 8, 1, 3, 2, 32),
    GBST_EQS(2, GBST_F32, true, 4, 2, 3, 1, 16),
    GBST_EQS(2, GBST_F32, true, 4, 2, 3, 1, 8),
    GBST_EQS(2, GBST_F32, true, 8, 2, 6, 1, 32),
    GBST_EQS(2, GBST_BF16, true, 4, 1, 3, 1, 16),
    GBST_EQS(2, GBST_BF16, true, 4, 1, 5, 2, 16),
    GBST_EQS(2, GBST_BF16, true, 4, 2, 3, 1, 16),
    GBST_EQS(2, GBST_BF16, true, 4, 1, 3, 1, 8),
    GBST_EQS(2, GBST_BF16, true, 8, 1, 3, 2, 16),
    GBST_EQS(2, GBST_BF16, true, 8, 1, 5, 2, 16),
};
}  // namespace

const Entry *table_r2(int *n)
{
    *n = static_cast<int>(sizeof(kTable) / sizeof(kTable[0]));
    return kTable;
}
}  // namespace sweep
}  // namespace gbst
