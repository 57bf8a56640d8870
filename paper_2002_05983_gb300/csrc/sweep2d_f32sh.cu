// Streaming-kernel instantiations with one coefficient per distance (shared
// coefficients), float storage; 2D, 128 threads x 4 cells per block row,
// radius 1..4 at the temporal degrees the full-coefficient defaults use.
#include "registry.h"
#include "sweep_kernel.cuh"

namespace stn {
namespace {
const KernelEntry kList[] = {
    STN_EX(2, 1, 1, 1, float, 0, 128, 1, true),
    STN_EX(2, 1, 2, 1, float, 0, 128, 1, true),
    STN_EX(2, 1, 3, 1, float, 0, 128, 1, true),
    STN_EX(2, 1, 4, 1, float, 0, 128, 1, true),
    STN_EX(2, 1, 5, 1, float, 0, 128, 1, true),
    STN_EX(2, 2, 1, 1, float, 0, 128, 1, true),
    STN_EX(2, 2, 2, 1, float, 0, 128, 1, true),
    STN_EX(2, 2, 3, 1, float, 0, 128, 1, true),
    STN_EX(2, 3, 1, 1, float, 0, 128, 1, true),
    STN_EX(2, 3, 2, 1, float, 0, 128, 1, true),
    STN_EX(2, 4, 1, 1, float, 0, 128, 1, true),
    STN_EX(2, 4, 2, 1, float, 0, 128, 1, true)};
}  // namespace
int list_2d_f32sh(const KernelEntry **e)
{
    *e = kList;
    return static_cast<int>(sizeof(kList) / sizeof(kList[0]));
}
}  // namespace stn
