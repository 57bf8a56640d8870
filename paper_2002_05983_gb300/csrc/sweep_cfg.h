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
// Steps loaded ahead by 3D radius-1 kernels of T levels with ES-byte storage.  FP32 rings
// of 64x16-cell tiles: t = 2 with 3 steps ahead (43.0 KB) keeps 5 blocks per SM instead
// of 4 (+9 % on 512^3), t >= 3 with 2 steps ahead keeps 4 instead of 3 (+6 %); one level
// keeps 4 steps (it is not limited by shared memory, and shorter steps need the
// deeper prefetch).  16-bit input rings are small enough at 4 steps.
__host__ __device__ constexpr int pf3r1(int t, int es) { return es != 4 || t <= 1 ? 4 : (t == 2 ? 3 : 2); }

__host__ __device__ constexpr int cdiv(int a, int b) { return (a + b - 1) / b; }
__host__ __device__ constexpr int rup(int a, int b) { return cdiv(a, b) * b; }

// D: 2 or 3; R: radius; T: time levels per pass; VY: y rows per thread (3D);
// ES: bytes per stored element (4 fp32, 2 bf16/fp16); TX x TY threads;
// P: planes every level advances per step (rows in 2D; 1 in 3D).
template <int D, int R, int T, int VY, int ES, int TX, int TY, int P = 1> struct Geo {
    static_assert(P == 1 || ((P == 2 || P == 4) && D == 2), "several planes per step are a 2D schedule");
    static constexpr bool F32S = ES == 4;
    static constexpr int NV = cdiv(R, 4);              // 4-cell vectors of x neighbours per side
    static constexpr int ALIGN = 16 / ES;              // cells per 16 bytes of storage
    static constexpr int PAD32 = 4 * NV;               // FP32 ring row padding (cells)
    static constexpr int BX = 4 * TX;                  // thread-region width (cells)
    static constexpr int BY = (D == 3) ? TY * VY : 1;  // thread-region rows (3D)
    // x halo of levels 1..T in whole 4-cell vectors.  Tile origins (multiples of CX) and the
    // input box origin gx0 - PADIN stay on 16-byte boundaries: CX = BX - 2*HTX is a multiple of
    // 8 cells, and the input padding (at least the 4*NV cells the neighbour loads reach) takes
    // 4 more cells where HTX + 4*NV is not a 16-byte multiple (16-bit storage only).
    static constexpr int HTX = rup((T - 1) * R, 4);
    static constexpr int PADIN = (HTX + 4 * NV) % ALIGN == 0 ? 4 * NV : 4 * NV + 4;   // input row padding
    static constexpr int HTY = (D == 3) ? (T - 1) * R : 0;
    static constexpr int CX = BX - 2 * HTX;            // compute tile (Eq. 2: bsize - 2 t r)
    static constexpr int CY = (D == 3) ? BY - 2 * HTY : 1;
    static constexpr int PW = BX + 2 * PAD32;          // FP32 plane row: PAD32 pad cells either side
    static constexpr int PH = (D == 3) ? BY + 2 * R : 1;
    static constexpr int PWIN = BX + 2 * PADIN;        // input plane row (elements)
    static constexpr int SLOT32 = rup(PW * PH, 32);    // floats per FP32 ring slot
    static constexpr int SLOTIN = rup(PWIN * PH * ES, 128) / ES;   // elements per input slot
    // Plane lags.  Level s handles planes P*k - lag(s) + j (j < P) at step k.  Level 1
    // trails the input by L1 >= R planes (its stream-axis neighbours are in registers) and
    // by >= P planes (the input planes it reads in shared memory had their clamp frame
    // written in an earlier step); each further level trails the one below by GAP = P +
    // max(R, P): the r planes ahead it needs were computed in an earlier step, and the
    // planes it reads in shared memory had their clamp frame filled an earlier step still.
    static constexpr int L1 = R > P ? R : P;
    static constexpr int GAP = P + L1;
    // A level's register queue (and FP32 ring) spans the GAP + R planes the level above
    // reads in one step, rounded up to whole steps: plane p sits in slot p mod QP.
    static constexpr int QP = rup(GAP + R, P);
    static constexpr int PFMIN = (D == 2) ? 4 : 2;     // planes loaded ahead at least
    // Steps per unrolled chunk.  The register queue of a level holds QP planes;
    // with U = QP / P steps per chunk it rotates through fixed registers (ROT).  In
    // 3D, a rotating chunk larger than kRotMaxFma misses the instruction cache, so
    // chunks of U < QP steps append to a queue of QP + U registers and shift it
    // down by U planes at the chunk's end (QP moves per cell and level every U
    // steps): measured 1.2-1.4x faster for 3D r = 3, 4.  2D keeps the rotating
    // queue at every size: there the moves cost more than the misses they avoid.
    static constexpr int BODY = T * VY * 4 * (2 * D * R + 1);
    static constexpr bool ROT = D == 2 || QP * BODY <= kRotMaxFma;
    static constexpr int U = ROT ? QP / P : (kChunkFma / BODY >= 1 ? kChunkFma / BODY : 1);
    static constexpr int NQ = ROT ? QP : QP + U;       // queue registers per level and cell
    // Input ring in steps of P planes: the step that level 1 reads in shared memory lags
    // the newest by KS = ceil(L1 / P) steps; PFS steps are loaded ahead.
    static constexpr int KS = cdiv(L1, P);
    // Step slots of the ring.  3D radius 1 keeps a rotating chunk of U = 3 steps, and a
    // ring rounded up to whole chunks would hold 6 slots; its ring holds KS + 1 + pf3r1
    // slots instead and, where that is not a chunk multiple, wraps inside a chunk
    // (run-time slot index per step, WRAP).
    static constexpr int DS = (D == 3 && ROT && R == 1) ? KS + 1 + pf3r1(T, ES)
                                                        : U * cdiv(KS + 1 + cdiv(PFMIN, P), U);
    static constexpr bool WRAP = DS % U != 0;
    static constexpr int PFS = DS - KS - 1;            // steps loaded ahead of use
    static constexpr int PF = P * PFS;                 // planes loaded ahead of use
    static constexpr int DEPTH = P * DS;               // input ring slots (planes)
    static constexpr int NRING = T - 1;                // FP32 rings written by levels 1..T-1
    static constexpr size_t SMEM = static_cast<size_t>(kSmemHeader) +
                                   static_cast<size_t>(DEPTH) * SLOTIN * ES +
                                   static_cast<size_t>(NRING) * QP * SLOT32 * 4;
    static_assert(BX % ALIGN == 0 && CX % ALIGN == 0 && (HTX + PADIN) % ALIGN == 0, "16-byte tile and box origins");
    static constexpr bool OK = CX >= 8 && CY >= 1 && DS <= kMaxDepthIn && U <= DS &&
                               (D == 2 || (PWIN <= 256 && PH <= 256));
    // plane lag of level s (plane p of level s is handled at step (p + lag(s)) / P)
    __host__ __device__ static constexpr int lag(int s) { return s == 0 ? 0 : L1 + (s - 1) * GAP; }
};

}  // namespace stn
