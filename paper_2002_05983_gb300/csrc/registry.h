// Table of compiled streaming-kernel instantiations (filled by sweep*_*.cu).
#pragma once
#include <cstddef>

#include "sweep_cfg.h"

namespace stn {

struct KernelEntry {
    int dim, r, t, vy, dtype;   // dtype: 0 fp32, 1 bf16, 2 fp16
    int sh;                     // bit 0: one coefficient per distance; bit 1: bounds-checked build
    int tx, ty;                 // block shape
    int p;                      // planes every level advances per step (2D rows: 1 or 2; 3D: 1)
    int qp, u, rot;             // register-queue period (planes), steps per unrolled chunk, rotating queue
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
int list_2d_f32_p2(const KernelEntry **e);
int list_2d_bf16_p2(const KernelEntry **e);
int list_2d_f16_p2(const KernelEntry **e);
int list_2d_p4(const KernelEntry **e);

}  // namespace stn

#define STN_G(D, R, T, VY, S, TX, TY, P) stn::Geo<D, R, T, VY, static_cast<int>(sizeof(S)), TX, TY, P>
#define STN_E(D, R, T, VY, S, DT, TX, TY) STN_EXC(D, R, T, VY, S, DT, TX, TY, false, false, 1)
#define STN_EP(D, R, T, S, DT, P) STN_EXC(D, R, T, 1, S, DT, 128, 1, false, false, P)
#define STN_EX(D, R, T, VY, S, DT, TX, TY, SH) STN_EXC(D, R, T, VY, S, DT, TX, TY, SH, false, 1)
// kind = SH + 2 * CHK: coefficient form and bounds-checked build; P planes per step
#define STN_EXC(D, R, T, VY, S, DT, TX, TY, SH, CHK, P)                                            \
    {D, R, T, VY, DT, (SH ? 1 : 0) + (CHK ? 2 : 0), TX, TY, P, STN_G(D, R, T, VY, S, TX, TY, P)::QP,  \
     STN_G(D, R, T, VY, S, TX, TY, P)::U, STN_G(D, R, T, VY, S, TX, TY, P)::ROT ? 1 : 0,              \
     STN_G(D, R, T, VY, S, TX, TY, P)::CX,                                                          \
     STN_G(D, R, T, VY, S, TX, TY, P)::CY,                                                          \
     STN_G(D, R, T, VY, S, TX, TY, P)::HTX, STN_G(D, R, T, VY, S, TX, TY, P)::HTY,                  \
     STN_G(D, R, T, VY, S, TX, TY, P)::PF, STN_G(D, R, T, VY, S, TX, TY, P)::PADIN,                 \
     STN_G(D, R, T, VY, S, TX, TY, P)::SMEM,                                                        \
     reinterpret_cast<const void *>(&stn::sweep_kernel<D, R, T, VY, S, TX, TY, SH, CHK, P>),         \
     reinterpret_cast<const void *>(&stn::sweep_persistent<D, R, T, VY, S, TX, TY, SH, CHK, P>)}
