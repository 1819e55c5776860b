// Variants whose x-neighbour sums of odd offsets (operands that straddle the
// thread's packed FP32x2 point pairs) are two scalar additions instead of one
// packed addition of re-paired registers: fewer instructions per point, the
// same results bit for bit.  The shapes are those the autotuner picks among the
// packed-only variants.  The BF16 wave variants also form their y-neighbour
// sums and 2u - u^{n-1} with mixed-precision (BF16 + FP32) additions, and the
// radius-1 two-step kernel gets a deeper prefetch.  A table of its own, after the
// others, so that the indices of the earlier variants stay as they were.
#include "sweep_tb.cuh"

namespace gbst {
namespace sweep {
namespace {
constexpr int kSX = kOptScalarOddX;
const Entry kTable[] = {
    // radius 4, 3D heat, FP32
    entry<4, GBST_HEAT, GBST_F32, true, 4, 2, 7, 2, 32, false, kSX>(),
    entry<4, GBST_HEAT, GBST_F32, true, 4, 2, 5, 2, 32, false, kSX>(),
    entry<4, GBST_HEAT, GBST_F32, true, 8, 2, 9, 1, 32, false, kSX>(),
    entry<4, GBST_HEAT, GBST_F32, true, 4, 2, 5, 2, 16, false, kSX>(),
    // radius 4, 3D wave, FP32 and BF16 storage
    entry<4, GBST_WAVE, GBST_F32, true, 8, 1, 3, 2, 32, false, kSX>(),
    entry<4, GBST_WAVE, GBST_BF16, true, 8, 1, 5, 1, 16, false, kSX>(),
    entry<4, GBST_WAVE, GBST_BF16, true, 8, 1, 3, 1, 16, false, kSX>(),
    // radius 4, 2D heat (128 x 32 tiles)
    entry<4, GBST_HEAT, GBST_F32, false, 4, 8, 2, 1, 32, false, kSX>(),
    // radius 2, 3D heat, four rows per thread
    entry<2, GBST_HEAT, GBST_F32, true, 4, 4, 3, 1, 32, false, kSX>(),
    entry<2, GBST_HEAT, GBST_F32, true, 4, 4, 3, 2, 32, false, kSX>(),
    // radius 1, two steps per launch
    tb_entry<1, 10, 4, 2, 1, kSX>(),
    tb_entry<1, 10, 3, 2, 1, kSX>(),
    // radius 4, 3D wave, BF16 storage, mixed-precision y sums and 2u - u^{n-1}: fewer
    // instructions per point, so more CTAs per SM pay (3 x 5 warps: 586 GPoints/s at 768^3
    // against 528 for one CTA of 9 warps without the mixed-precision forms)
    entry<4, GBST_WAVE, GBST_BF16, true, 8, 1, 5, 1, 16, false, kSX | kOptMixedY | kOptMixedU>(),
    entry<4, GBST_WAVE, GBST_BF16, true, 4, 1, 5, 2, 16, false, kSX | kOptMixedY | kOptMixedU>(),
    entry<4, GBST_WAVE, GBST_BF16, true, 4, 1, 7, 2, 16, false, kSX | kOptMixedY | kOptMixedU>(),
    entry<4, GBST_WAVE, GBST_BF16, true, 4, 1, 3, 3, 16, false, kSX | kOptMixedY | kOptMixedU>(),
    entry<4, GBST_WAVE, GBST_BF16, true, 4, 1, 4, 3, 16, false, kSX | kOptMixedY | kOptMixedU>(),
    // radius 1, two steps per launch, three planes in flight
    tb_entry<1, 10, 3, 3, 1, kSX>(),
};
}  // namespace

const Entry *table_sx(int *n)
{
    *n = static_cast<int>(sizeof(kTable) / sizeof(kTable[0]));
    return kTable;
}
}  // namespace sweep
}  // namespace gbst
