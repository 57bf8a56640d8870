// Table of compiled streaming-kernel instantiations (filled by sweep*_*.cu).
#pragma once
#include <cstddef>

#include "sweep_cfg.h"

namespace stn {

struct KernelEntry {
    int dim, r, t, vy, dtype;   // dtype: 0 fp32, 1 bf16, 2 fp16
    int sh;                     // bit 0: one coefficient per distance; bit 1: bounds-checked build
    int tx, ty;                 // block shape
    int cx, cy, htx, hty;       // compute tile and thread-region halo
    int pf;                     // planes loaded ahead of use
    int padin;                  // input-plane x padding per side (cells): TMA box width 4*tx + 2*padin
    size_t smem;                // dynamic shared memory bytes
    const void *fn;             // __global__ sweep_kernel<dim, r, t, vy, S, tx, ty>
    const void *pfn;            // __global__ sweep_persistent<dim, r, t, vy, S, tx, ty>
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
int list_2d_f32_r5(const KernelEntry **e);
int list_2d_f32_r6(const KernelEntry **e);
int list_3d_f32_r5(const KernelEntry **e);
int list_3d_f32_r6(const KernelEntry **e);
int list_2d_bf16_r5(const KernelEntry **e);
int list_2d_bf16_r6(const KernelEntry **e);
int list_3d_bf16_r5(const KernelEntry **e);
int list_3d_bf16_r6(const KernelEntry **e);
int list_2d_f16_r5(const KernelEntry **e);
int list_2d_f16_r6(const KernelEntry **e);
int list_3d_f16_r5(const KernelEntry **e);
int list_3d_f16_r6(const KernelEntry **e);
int list_2d_f32sh(const KernelEntry **e);
int list_3d_f32sh(const KernelEntry **e);
int list_checked(const KernelEntry **e);

}  // namespace stn

#define STN_G(D, R, T, VY, S, TX, TY) stn::Geo<D, R, T, VY, static_cast<int>(sizeof(S)), TX, TY>
#define STN_E(D, R, T, VY, S, DT, TX, TY) STN_EXC(D, R, T, VY, S, DT, TX, TY, false, false)
#define STN_EX(D, R, T, VY, S, DT, TX, TY, SH) STN_EXC(D, R, T, VY, S, DT, TX, TY, SH, false)
// kind = SH + 2 * CHK: coefficient form and bounds-checked build
#define STN_EXC(D, R, T, VY, S, DT, TX, TY, SH, CHK)                                               \
    {D, R, T, VY, DT, (SH ? 1 : 0) + (CHK ? 2 : 0), TX, TY, STN_G(D, R, T, VY, S, TX, TY)::CX,        \
     STN_G(D, R, T, VY, S, TX, TY)::CY,                                                             \
     STN_G(D, R, T, VY, S, TX, TY)::HTX, STN_G(D, R, T, VY, S, TX, TY)::HTY,                        \
     STN_G(D, R, T, VY, S, TX, TY)::PF, STN_G(D, R, T, VY, S, TX, TY)::PADIN,                       \
     STN_G(D, R, T, VY, S, TX, TY)::SMEM,                                                             \
     reinterpret_cast<const void *>(&stn::sweep_kernel<D, R, T, VY, S, TX, TY, SH, CHK>),            \
     reinterpret_cast<const void *>(&stn::sweep_persistent<D, R, T, VY, S, TX, TY, SH, CHK>)}
