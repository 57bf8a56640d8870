// One thread per cell, one time step per launch: the plain form of Eq. 1
// with clamp-to-edge loads.  It is the t = 1 reference schedule that the
// streaming kernel must match bit for bit, and the path for grids whose rows
// are not 16-byte aligned (the streaming kernel's copies need aligned rows).
#include "naive.h"

namespace stn {
namespace {

template <typename S> __device__ __forceinline__ float ld1(const S *p);
template <> __device__ __forceinline__ float ld1<float>(const float *p) { return *p; }
template <> __device__ __forceinline__ float ld1<__nv_bfloat16>(const __nv_bfloat16 *p)
{
    return __bfloat162float(*p);
}
template <> __device__ __forceinline__ float ld1<__half>(const __half *p) { return __half2float(*p); }

template <typename S> __device__ __forceinline__ S st1(float v);
template <> __device__ __forceinline__ float st1<float>(float v) { return v; }
template <> __device__ __forceinline__ __nv_bfloat16 st1<__nv_bfloat16>(float v)
{
    return __float2bfloat16_rn(v);
}
template <> __device__ __forceinline__ __half st1<__half>(float v) { return __float2half_rn(v); }

// SH: one coefficient per distance; the 2*D neighbours at distance i are summed
// left to right (W, E, S, N[, B, A]) and then enter one FMA.
template <int D, int R, typename S, bool SH>
__global__ void __launch_bounds__(256)
    naive_kernel(const S *__restrict__ in, S *__restrict__ out, const __grid_constant__ NaiveArgs a)
{
    const int64_t n = static_cast<int64_t>(a.nx) * a.ny * a.nz;
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t idx = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; idx < n;
         idx += stride) {
        const int x = static_cast<int>(idx % a.nx);
        const int64_t rest = idx / a.nx;
        const int y = static_cast<int>(rest % a.ny);
        const int z = static_cast<int>(rest / a.ny);
        auto at = [&](int xx, int yy, int zz) {
            return ld1<S>(in + (static_cast<int64_t>(zz) * a.ny + yy) * a.nx + xx);
        };
        float acc = __fmul_rn(a.c[0], at(x, y, z));
#pragma unroll
        for (int i = 1; i <= R; ++i) {
            if constexpr (SH) {
                float sum = __fadd_rn(at(max(x - i, 0), y, z), at(min(x + i, a.nx - 1), y, z));
                sum = __fadd_rn(sum, at(x, max(y - i, 0), z));
                sum = __fadd_rn(sum, at(x, min(y + i, a.ny - 1), z));
                if (D == 3) {
                    sum = __fadd_rn(sum, at(x, y, max(z - i, 0)));
                    sum = __fadd_rn(sum, at(x, y, min(z + i, a.nz - 1)));
                }
                acc = __fmaf_rn(a.c[i], sum, acc);
                continue;
            }
            const int cb = 1 + (i - 1) * 2 * D;
            acc = __fmaf_rn(a.c[cb + 0], at(max(x - i, 0), y, z), acc);
            acc = __fmaf_rn(a.c[cb + 1], at(min(x + i, a.nx - 1), y, z), acc);
            acc = __fmaf_rn(a.c[cb + 2], at(x, max(y - i, 0), z), acc);
            acc = __fmaf_rn(a.c[cb + 3], at(x, min(y + i, a.ny - 1), z), acc);
            if (D == 3) {
                acc = __fmaf_rn(a.c[cb + 4], at(x, y, max(z - i, 0)), acc);
                acc = __fmaf_rn(a.c[cb + 5], at(x, y, min(z + i, a.nz - 1)), acc);
            }
        }
        out[idx] = st1<S>(acc);
    }
}

template <int D, int R, bool SH>
const void *pick_sh(int dtype)
{
    switch (dtype) {
    case 0: return reinterpret_cast<const void *>(&naive_kernel<D, R, float, SH>);
    case 1: return reinterpret_cast<const void *>(&naive_kernel<D, R, __nv_bfloat16, SH>);
    case 2: return reinterpret_cast<const void *>(&naive_kernel<D, R, __half, SH>);
    default: return nullptr;
    }
}

template <int D, int R>
const void *pick(int dtype, int sh)
{
    return sh ? pick_sh<D, R, true>(dtype) : pick_sh<D, R, false>(dtype);
}

}  // namespace

const void *naive_fn(int dim, int r, int dtype, int sh)
{
    if (dim == 2) {
        switch (r) {
        case 1: return pick<2, 1>(dtype, sh);
        case 2: return pick<2, 2>(dtype, sh);
        case 3: return pick<2, 3>(dtype, sh);
        case 4: return pick<2, 4>(dtype, sh);
        case 5: return pick<2, 5>(dtype, sh);
        case 6: return pick<2, 6>(dtype, sh);
        }
    } else if (dim == 3) {
        switch (r) {
        case 1: return pick<3, 1>(dtype, sh);
        case 2: return pick<3, 2>(dtype, sh);
        case 3: return pick<3, 3>(dtype, sh);
        case 4: return pick<3, 4>(dtype, sh);
        case 5: return pick<3, 5>(dtype, sh);
        case 6: return pick<3, 6>(dtype, sh);
        }
    }
    return nullptr;
}

}  // namespace stn
