// Streaming-kernel instantiations: radius 6, __nv_bfloat16 storage;
// 2D, 128 threads x 4 cells per block row, temporal degrees 1..3.
#include "registry.h"
#include "sweep_kernel.cuh"

namespace stn {
namespace {
const KernelEntry kList[] = {
    STN_E(2, 6, 1, 1, __nv_bfloat16, 1, 128, 1),
    STN_E(2, 6, 2, 1, __nv_bfloat16, 1, 128, 1),
    STN_E(2, 6, 3, 1, __nv_bfloat16, 1, 128, 1)};
}  // namespace
int list_2d_bf16_r6(const KernelEntry **e)
{
    *e = kList;
    return static_cast<int>(sizeof(kList) / sizeof(kList[0]));
}
}  // namespace stn
