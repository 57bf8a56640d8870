// Compile-time geometry of one streaming-kernel instantiation, shared by the
// kernel and the host planner so both agree on tiles, halos and shared memory.
#pragma once
#include <cstddef>

namespace stn {

constexpr int kMaxR = 6;             // largest radius
constexpr int kMaxK = 2 * 3 * kMaxR + 1;   // coefficients of a 3D radius-6 stencil
constexpr int kSmemHeader = 1024;    // mbarriers + abort flag
constexpr int kMaxDepthIn = 64;
constexpr unsigned kStatusTimeout = 1u;
constexpr unsigned kStatusBounds = 2u;   // a bounds-checked kernel found an access out of range
// Unrolled-chunk sizes in FMA per thread (steps x levels x cells x (2*D*r+1)):
// 3D kernels whose rotating chunk exceeds kRotMaxFma use shifting chunks of about
// kChunkFma (see Geo::U).
constexpr int kRotMaxFma = 600;
constexpr int kChunkFma = 300;

__host__ __device__ constexpr int cdiv(int a, int b) { return (a + b - 1) / b; }
__host__ __device__ constexpr int rup(int a, int b) { return cdiv(a, b) * b; }

// D: 2 or 3; R: radius; T: time levels per pass; VY: y rows per thread (3D);
// ES: bytes per stored element (4 fp32, 2 bf16/fp16); TX x TY threads.
template <int D, int R, int T, int VY, int ES, int TX, int TY> struct Geo {
    static constexpr int QP = 2 * R + 1;               // register-queue period
    static constexpr bool F32S = ES == 4;
    static constexpr int NV = cdiv(R, 4);              // 4-cell vectors of x neighbours per side
    static constexpr int ALIGN = 16 / ES;              // cells per 16 bytes of storage
    static constexpr int PADIN = ALIGN > 4 * NV ? ALIGN : 4 * NV;   // input row padding (cells)
    static constexpr int PAD32 = 4 * NV;               // FP32 ring row padding (cells)
    static constexpr int BX = 4 * TX;                  // thread-region width (cells)
    static constexpr int BY = (D == 3) ? TY * VY : 1;  // thread-region rows (3D)
    static constexpr int HTX = rup((T - 1) * R, ALIGN);   // x halo of levels 1..T (16-byte multiple)
    static constexpr int HTY = (D == 3) ? (T - 1) * R : 0;
    static constexpr int CX = BX - 2 * HTX;            // compute tile (Eq. 2: bsize - 2 t r)
    static constexpr int CY = (D == 3) ? BY - 2 * HTY : 1;
    static constexpr int PW = BX + 2 * PAD32;          // FP32 plane row: PAD32 pad cells either side
    static constexpr int PH = (D == 3) ? BY + 2 * R : 1;
    static constexpr int PWIN = BX + 2 * PADIN;        // input plane row (elements)
    static constexpr int SLOT32 = rup(PW * PH, 32);    // floats per FP32 ring slot
    static constexpr int SLOTIN = rup(PWIN * PH * ES, 128) / ES;   // elements per input slot
    static constexpr int PFMIN = (D == 2) ? 4 : 2;
    // Steps per unrolled chunk.  The register queue of a level holds 2r+1 planes;
    // with U = QP steps per chunk it rotates through fixed registers (ROT).  In
    // 3D, a rotating chunk larger than kRotMaxFma misses the instruction cache, so
    // chunks of U < QP steps append to a queue of QP + U registers and shift it
    // down by U planes at the chunk's end (QP moves per cell and level every U
    // steps): measured 1.2-1.4x faster for 3D r = 3, 4.  2D keeps the rotating
    // queue at every size: there the moves cost more than the misses they avoid.
    static constexpr int BODY = T * VY * 4 * (2 * D * R + 1);
    static constexpr bool ROT = D == 2 || QP * BODY <= kRotMaxFma;
    static constexpr int U = ROT ? QP : (kChunkFma / BODY >= 1 ? kChunkFma / BODY : 1);
    static constexpr int NQ = ROT ? QP : QP + U;       // queue registers per level and cell
    static constexpr int LAG1 = R;                     // steps level 1 trails the input
    static constexpr int KEEP = R + 1;                 // input slots held besides prefetch
    static constexpr int DEPTH = U * cdiv(KEEP + PFMIN, U);     // input ring slots (chunk multiple)
    static constexpr int PF = DEPTH - KEEP;            // planes loaded ahead of use
    static constexpr int NRING = T - 1;                // FP32 rings written by levels 1..T-1
    static constexpr size_t SMEM = static_cast<size_t>(kSmemHeader) +
                                   static_cast<size_t>(DEPTH) * SLOTIN * ES +
                                   static_cast<size_t>(NRING) * QP * SLOT32 * 4;
    static constexpr bool OK = CX >= 8 && CY >= 1 && DEPTH <= kMaxDepthIn &&
                               (D == 2 || (PWIN <= 256 && PH <= 256));
    // step at which level s handles plane p: p + lag(s)
    __host__ __device__ static constexpr int lag(int s) { return s == 0 ? 0 : LAG1 + (s - 1) * (R + 1); }
};

}  // namespace stn
