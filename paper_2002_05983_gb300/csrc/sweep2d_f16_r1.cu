// Streaming-kernel instantiations: radius 1, __half storage;
// 2D, 128 threads x 4 cells per block row, every temporal degree whose register queue ((2r+1) rows x 4 cells x t levels) fits.
#include "registry.h"
#include "sweep_kernel.cuh"

namespace stn {
namespace {
const KernelEntry kList[] = {
    STN_E(2, 1, 1, 1, __half, 2, 128, 1),
    STN_E(2, 1, 2, 1, __half, 2, 128, 1),
    STN_E(2, 1, 3, 1, __half, 2, 128, 1),
    STN_E(2, 1, 4, 1, __half, 2, 128, 1),
    STN_E(2, 1, 5, 1, __half, 2, 128, 1),
    STN_E(2, 1, 6, 1, __half, 2, 128, 1),
    STN_E(2, 1, 7, 1, __half, 2, 128, 1),
    STN_E(2, 1, 8, 1, __half, 2, 128, 1),
    STN_E(2, 1, 9, 1, __half, 2, 128, 1),
    STN_E(2, 1, 10, 1, __half, 2, 128, 1),
    STN_E(2, 1, 11, 1, __half, 2, 128, 1),
    STN_E(2, 1, 12, 1, __half, 2, 128, 1),
    STN_E(2, 1, 13, 1, __half, 2, 128, 1),
    STN_E(2, 1, 14, 1, __half, 2, 128, 1),
    STN_E(2, 1, 15, 1, __half, 2, 128, 1),
    STN_E(2, 1, 16, 1, __half, 2, 128, 1)};
}  // namespace
int list_2d_f16_r1(const KernelEntry **e)
{
    *e = kList;
    return static_cast<int>(sizeof(kList) / sizeof(kList[0]));
}
}  // namespace stn
