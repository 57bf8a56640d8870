// Streaming-kernel instantiations: BF16 storage, 2D, 128 threads x 4 cells per block row,
// two rows per step (every level advances two rows between barriers, so the per-step
// bookkeeping, copy wait and barrier are shared by two rows).
#include "registry.h"
#include "sweep_kernel.cuh"

namespace stn {
namespace {
const KernelEntry kList[] = {
    STN_EP(2, 1, 1, __nv_bfloat16, 1, 2),
    STN_EP(2, 1, 2, __nv_bfloat16, 1, 2),
    STN_EP(2, 1, 3, __nv_bfloat16, 1, 2),
    STN_EP(2, 1, 4, __nv_bfloat16, 1, 2),
    STN_EP(2, 2, 1, __nv_bfloat16, 1, 2),
    STN_EP(2, 2, 2, __nv_bfloat16, 1, 2),
    STN_EP(2, 2, 3, __nv_bfloat16, 1, 2),
    STN_EP(2, 3, 1, __nv_bfloat16, 1, 2),
    STN_EP(2, 3, 2, __nv_bfloat16, 1, 2),
    STN_EP(2, 3, 3, __nv_bfloat16, 1, 2),
    STN_EP(2, 4, 1, __nv_bfloat16, 1, 2),
    STN_EP(2, 4, 2, __nv_bfloat16, 1, 2),
    STN_EP(2, 4, 3, __nv_bfloat16, 1, 2)};
}  // namespace
int list_2d_bf16_p2(const KernelEntry **e)
{
    *e = kList;
    return static_cast<int>(sizeof(kList) / sizeof(kList[0]));
}
}  // namespace stn
