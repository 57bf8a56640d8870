// Streaming-kernel instantiations: radius 4, __half storage;
// 3D, 16 x 8 threads, 2 or 4 y rows per thread, every temporal degree whose register queue fits.
#include "registry.h"
#include "sweep_kernel.cuh"

namespace stn {
namespace {
const KernelEntry kList[] = {
    STN_E(3, 4, 1, 2, __half, 2, 16, 8),
    STN_E(3, 4, 2, 2, __half, 2, 16, 8),
    STN_E(3, 4, 1, 4, __half, 2, 16, 8)};
}  // namespace
int list_3d_f16_r4(const KernelEntry **e)
{
    *e = kList;
    return static_cast<int>(sizeof(kList) / sizeof(kList[0]));
}
}  // namespace stn
