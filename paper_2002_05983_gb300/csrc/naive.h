#pragma once
#include <cstdint>

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "sweep_cfg.h"

namespace stn {

struct NaiveArgs {
    int nx, ny, nz;
    float c[kMaxK];
};

// __global__ naive_kernel<dim, r, S, sh>(const S* in, S* out, NaiveArgs) for dtype 0/1/2, or
// nullptr; sh = 1: one coefficient per distance.
const void *naive_fn(int dim, int r, int dtype, int sh);

}  // namespace stn
