// Table of compiled streaming-kernel instantiations (filled by sweep*_*.cu).
#pragma once

namespace stn {

struct KernelEntry {
    int dim, r, t, vy, dtype;   // dtype: 0 fp32, 1 bf16, 2 fp16
    const void *fn;             // __global__ sweep_kernel<dim, r, t, vy, S>
};

int list_2d_f32_r1(const KernelEntry **e);
int list_2d_f32_r2(const KernelEntry **e);
int list_2d_f32_r3(const KernelEntry **e);
int list_2d_f32_r4(const KernelEntry **e);
int list_3d_f32_r1(const KernelEntry **e);
int list_3d_f32_r2(const KernelEntry **e);
int list_3d_f32_r3(const KernelEntry **e);
int list_3d_f32_r4(const KernelEntry **e);
int list_2d_bf16_r1(const KernelEntry **e);
int list_2d_bf16_r2(const KernelEntry **e);
int list_2d_bf16_r3(const KernelEntry **e);
int list_2d_bf16_r4(const KernelEntry **e);
int list_3d_bf16_r1(const KernelEntry **e);
int list_3d_bf16_r2(const KernelEntry **e);
int list_3d_bf16_r3(const KernelEntry **e);
int list_3d_bf16_r4(const KernelEntry **e);
int list_2d_f16_r1(const KernelEntry **e);
int list_2d_f16_r2(const KernelEntry **e);
int list_2d_f16_r3(const KernelEntry **e);
int list_2d_f16_r4(const KernelEntry **e);
int list_3d_f16_r1(const KernelEntry **e);
int list_3d_f16_r2(const KernelEntry **e);
int list_3d_f16_r3(const KernelEntry **e);
int list_3d_f16_r4(const KernelEntry **e);

}  // namespace stn

#define STN_E(D, R, T, VY, S, DT) {D, R, T, VY, DT, reinterpret_cast<const void *>(&stn::sweep_kernel<D, R, T, VY, S>)}
