// Streaming-kernel instantiations: radius 5, __half storage;
// 3D, 16 x 8 threads, 2 or 4 y rows per thread, temporal degree 1 (a radius-5
// halo leaves too small a tile for more).
#include "registry.h"
#include "sweep_kernel.cuh"

namespace stn {
namespace {
const KernelEntry kList[] = {
    STN_E(3, 5, 1, 2, __half, 2, 16, 8),
    STN_E(3, 5, 1, 4, __half, 2, 16, 8)};
}  // namespace
int list_3d_f16_r5(const KernelEntry **e)
{
    *e = kList;
    return static_cast<int>(sizeof(kList) / sizeof(kList[0]));
}
}  // namespace stn
