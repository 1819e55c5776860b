// Streaming-sweep variants of radius 4 (space order 8), 2D grids: tiles, and
// one-row tiles streamed along y.  The first entry matching a grid's (equation,
// storage) is its default.
#include "sweep_stream.cuh"

namespace gbst {
namespace sweep {
namespace {
const Entry kTable[] = {
    GBST_EQS(4, GBST_F32, false, 4, 2, 3, 1, 16),
    GBST_EQS(4, GBST_F32, false, 4, 2, 3, 1, 32),
    GBST_EQS(4, GBST_F32, false, 4, 2, 5, 2, 32),
    GBST_EQS(4, GBST_F32, false, 4, 2, 3, 1, 8),
    GBST_EQS(4, GBST_F32, false, 4, 4, 3, 2, 32),
    GBST_EQS(4, GBST_F32, false, 8, 4, 2, 1, 32),
    GBST_EQS(4, GBST_F32, false, 4, 8, 2, 1, 32),
    GBST_EQS(4, GBST_BF16, false, 4, 1, 3, 1, 16),
    GBST_EQS(4, GBST_BF16, false, 4, 1, 3, 1, 8),
    GBST_EQS_YS(4, GBST_F32, 4, 8),
    GBST_EQS_YS(4, GBST_F32, 6, 8),
    GBST_EQS_YS(4, GBST_F32, 3, 12),
};
}  // namespace

const Entry *table_r4_2d(int *n)
{
    *n = static_cast<int>(sizeof(kTable) / sizeof(kTable[0]));
    return kTable;
}
}  // namespace sweep
}  // namespace gbst
