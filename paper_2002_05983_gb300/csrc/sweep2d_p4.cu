// Streaming-kernel instantiations: 2D, 128 threads x 4 cells per block row, one time level
// per pass (t = 1) with four rows per step, every storage type: the pass that 16-bit storage
// runs at, where the per-step bookkeeping is shared by four rows.
#include "registry.h"
#include "sweep_kernel.cuh"

namespace stn {
namespace {
const KernelEntry kList[] = {
    STN_EP(2, 1, 1, float, 0, 4),
    STN_EP(2, 2, 1, float, 0, 4),
    STN_EP(2, 3, 1, float, 0, 4),
    STN_EP(2, 4, 1, float, 0, 4),
    STN_EP(2, 1, 1, __nv_bfloat16, 1, 4),
    STN_EP(2, 2, 1, __nv_bfloat16, 1, 4),
    STN_EP(2, 3, 1, __nv_bfloat16, 1, 4),
    STN_EP(2, 4, 1, __nv_bfloat16, 1, 4),
    STN_EP(2, 1, 1, __half, 2, 4),
    STN_EP(2, 2, 1, __half, 2, 4),
    STN_EP(2, 3, 1, __half, 2, 4),
    STN_EP(2, 4, 1, __half, 2, 4)};
}  // namespace
int list_2d_p4(const KernelEntry **e)
{
    *e = kList;
    return static_cast<int>(sizeof(kList) / sizeof(kList[0]));
}
}  // namespace stn
