// Bounds-checked streaming-kernel instantiations (stencil_set_checked): every shared-memory
// access, global store and copy is range-checked and a violation is reported in the device
// status instead of being performed.  A few configurations that cover both dimensions, both
// storage widths, both register-queue forms, radii that need one and two neighbour vectors,
// temporal blocking and both block orders.
#include "registry.h"
#include "sweep_kernel.cuh"

namespace stn {
namespace {
const KernelEntry kList[] = {
    STN_EXC(2, 1, 1, 1, float, 0, 128, 1, false, true, 1),
    STN_EXC(2, 1, 5, 1, float, 0, 128, 1, false, true, 1),
    STN_EXC(2, 4, 2, 1, float, 0, 128, 1, false, true, 1),
    STN_EXC(2, 6, 2, 1, float, 0, 128, 1, false, true, 1),
    STN_EXC(2, 2, 3, 1, __nv_bfloat16, 1, 128, 1, false, true, 1),
    STN_EXC(3, 1, 2, 2, float, 0, 16, 8, false, true, 1),
    STN_EXC(3, 3, 1, 4, float, 0, 16, 8, false, true, 1),
    STN_EXC(3, 5, 1, 2, float, 0, 16, 8, false, true, 1),
    STN_EXC(3, 2, 1, 2, __half, 2, 16, 8, false, true, 1)};
}  // namespace
int list_checked(const KernelEntry **e)
{
    *e = kList;
    return static_cast<int>(sizeof(kList) / sizeof(kList[0]));
}
}  // namespace stn
