// Streaming-kernel instantiations with one coefficient per distance (shared
// coefficients), float storage; 3D, 16 x 8 threads, 2 y rows per thread.
#include "registry.h"
#include "sweep_kernel.cuh"

namespace stn {
namespace {
const KernelEntry kList[] = {
    STN_EX(3, 1, 1, 2, float, 0, 16, 8, true),
    STN_EX(3, 1, 2, 2, float, 0, 16, 8, true),
    STN_EX(3, 2, 1, 2, float, 0, 16, 8, true),
    STN_EX(3, 3, 1, 2, float, 0, 16, 8, true),
    STN_EX(3, 4, 1, 2, float, 0, 16, 8, true)};
}  // namespace
int list_3d_f32sh(const KernelEntry **e)
{
    *e = kList;
    return static_cast<int>(sizeof(kList) / sizeof(kList[0]));
}
}  // namespace stn
