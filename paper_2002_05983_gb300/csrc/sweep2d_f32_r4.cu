// Streaming-kernel instantiations: radius 4, float storage;
// 2D, 128 threads x 4 cells per block row, every temporal degree whose register queue ((2r+1) rows x 4 cells x t levels) fits.
#include "registry.h"
#include "sweep_kernel.cuh"

namespace stn {
namespace {
const KernelEntry kList[] = {
    STN_E(2, 4, 1, 1, float, 0, 128, 1),
    STN_E(2, 4, 2, 1, float, 0, 128, 1),
    STN_E(2, 4, 3, 1, float, 0, 128, 1),
    STN_E(2, 4, 4, 1, float, 0, 128, 1)};
}  // namespace
int list_2d_f32_r4(const KernelEntry **e)
{
    *e = kList;
    return static_cast<int>(sizeof(kList) / sizeof(kList[0]));
}
}  // namespace stn
