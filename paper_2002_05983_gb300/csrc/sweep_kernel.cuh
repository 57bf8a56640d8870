// Streaming star-stencil sweep for sm_103a: spatial blocking (1.5D in 2D,
// 2.5D in 3D) combined with overlapped temporal blocking of degree T
// (Sections III.A/III.B of the paper; Eq. 2 gives the shrinking valid
// region, csize = bsize - 2*T*r).
//
// One block owns a tile of the plane perpendicular to the streaming axis
// (2D: a run of x columns, streaming along y; 3D: an x/y tile, streaming
// along z) and a segment of the streaming axis.  Each step of the block's
// loop advances every time level by one plane:
//   * level 0 is the input: planes arrive by TMA (1D bulk copies of a row in
//     2D, a 3D tensor-map box in 3D) into a ring of shared-memory slots in
//     the storage type (FP32, BF16 or FP16) with one mbarrier per slot,
//     `prefetch` planes ahead of use;
//   * level s (1..T) computes plane k - lag(s), lag(s) = r + (s-1)*(r+1),
//     from level s-1: the streaming-axis neighbours come from a register
//     queue of 2r+1 planes of the thread's own cells, the in-plane
//     neighbours from shared memory (level 1 from the input ring, widened to
//     FP32 on load, which is exact; higher levels from FP32 rings of 2r+1
//     planes).  Everything a level reads in shared memory was written at
//     least one step earlier and is overwritten at least one step after its
//     last read, so one __syncthreads per step orders all of it; levels run
//     from T down to 2, then 0, then 1, so a level reads its register queue
//     before the level below overwrites the oldest plane of it;
//   * level T writes the compute tile of its plane to global memory.
// The FP32 arithmetic of every cell is one multiply and 2*D*r fused
// multiply-adds in the order centre, then for i = 1..r: W, E, S, N[, B, A]
// (Eq. 1 read left to right), so results do not depend on T, tiles or
// launch shape.
//
// Clamp to edge (Section III.B) at every time level: a plane segment that
// streams off the grid's end keeps repeating the last plane (queue copy); a
// segment that starts at plane 0 fills the whole queue with plane 0; in the
// plane, tiles at the grid's edge overwrite the out-of-grid frame of every
// level's ring plane with the clamped border values before anyone reads it.
#pragma once

#include <cstdint>
#include <type_traits>

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "sweep_cfg.h"

namespace stn {

constexpr int kMaxThreads = 256;

struct SweepArgs {
    const void *in;       // source grid (the 2D path reads rows with bulk copies)
    void *out;            // destination grid
    unsigned *status;     // sticky device status word
    int nx, ny, nz;       // grid extents (2D: nz = 1)
    int ns;               // extent of the streaming axis (2D: ny, 3D: nz)
    int seg;              // stream-axis rows/planes per block
    int flat;             // 1: blocks split the tile columns laid end to end; 0: slabs of seg planes
    int ntx, nty;         // tile counts in x and y (nty = 1 in 2D)
    int timeout_ms;       // limit of every bounded wait
    int fault_plane;      // test hook: never load this input plane (< 0: off)
    float c[kMaxK];       // coefficients, Eq. 1 order
    alignas(8) float cc[2 * kMaxK];   // each coefficient twice: the operand pairs of the packed two-lane FMAs
};

// --------------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait on an mbarrier phase: false after `timeout_ms` without completion.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, int timeout_ms)
{
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    const uint64_t lim = static_cast<uint64_t>(timeout_ms) * 1000000ull;
    while (!mbar_try_wait(bar, parity)) {
        if (global_ns() - t0 > lim) return false;
    }
    return true;
}

__device__ __forceinline__ void bulk_load(uint32_t dst, const void *src, uint32_t bytes,
                                          uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            dst),
        "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap *map, int x, int y,
                                            int z, uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
        : "memory");
}

// Packed two-lane FP32 arithmetic (sm_100 and later): two cells' chains advance in one
// instruction, each lane an IEEE multiply or fused multiply-add of its own, so a cell's
// value is the same as with scalar instructions in the same order.
__device__ __forceinline__ uint64_t pk2(float a, float b)
{
    uint64_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void upk2(uint64_t r, float &a, float &b)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r));
}
__device__ __forceinline__ uint64_t mul2(uint64_t a, uint64_t b)
{
    uint64_t d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ uint64_t fma2(uint64_t a, uint64_t b, uint64_t c)
{
    uint64_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

// --------------------------------------------------------- storage formats
template <typename S> struct Fmt;
template <> struct Fmt<float> {
    static constexpr int pad = 4;   // 16 bytes of padding either side of a row
    __device__ __forceinline__ static void load4(const float *p, float (&v)[4])
    {
        const float4 t = *reinterpret_cast<const float4 *>(p);
        v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
    }
    __device__ __forceinline__ static void store4(float *p, const float (&v)[4])
    {
        *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
    }
};
template <> struct Fmt<__nv_bfloat16> {
    static constexpr int pad = 8;
    __device__ __forceinline__ static void load4(const __nv_bfloat16 *p, float (&v)[4])
    {
        // a BF16 value is the upper half of the binary32 with the same bits: the lower cell of
        // each 32-bit pair moves up by 16 bits, the upper one keeps its place (exact)
        const uint2 t = *reinterpret_cast<const uint2 *>(p);
        v[0] = __uint_as_float(t.x << 16);
        v[1] = __uint_as_float(t.x & 0xffff0000u);
        v[2] = __uint_as_float(t.y << 16);
        v[3] = __uint_as_float(t.y & 0xffff0000u);
    }
    __device__ __forceinline__ static void store4(__nv_bfloat16 *p, const float (&v)[4])
    {
        __nv_bfloat162 a = __floats2bfloat162_rn(v[0], v[1]);
        __nv_bfloat162 b = __floats2bfloat162_rn(v[2], v[3]);
        uint2 t;
        t.x = *reinterpret_cast<uint32_t *>(&a);
        t.y = *reinterpret_cast<uint32_t *>(&b);
        *reinterpret_cast<uint2 *>(p) = t;
    }
};
template <> struct Fmt<__half> {
    static constexpr int pad = 8;
    __device__ __forceinline__ static void load4(const __half *p, float (&v)[4])
    {
        const uint2 t = *reinterpret_cast<const uint2 *>(p);
        const float2 a = __half22float2(*reinterpret_cast<const __half2 *>(&t.x));
        const float2 b = __half22float2(*reinterpret_cast<const __half2 *>(&t.y));
        v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
    }
    __device__ __forceinline__ static void store4(__half *p, const float (&v)[4])
    {
        __half2 a = __floats2half2_rn(v[0], v[1]);
        __half2 b = __floats2half2_rn(v[2], v[3]);
        uint2 t;
        t.x = *reinterpret_cast<uint32_t *>(&a);
        t.y = *reinterpret_cast<uint32_t *>(&b);
        *reinterpret_cast<uint2 *>(p) = t;
    }
};

// ------------------------------------------------------ compile-time loops
template <int I> using IC = std::integral_constant<int, I>;
template <int I, int N> struct SFor {
    template <typename F> __device__ __forceinline__ static void run(F &&f)
    {
        f(IC<I>{});
        SFor<I + 1, N>::run(f);
    }
};
template <int N> struct SFor<N, N> {
    template <typename F> __device__ __forceinline__ static void run(F &&) {}
};

__host__ __device__ constexpr int cmod(int a, int m) { return ((a % m) + m) % m; }
__host__ __device__ constexpr int cclamp(int a, int lo, int hi) { return a < lo ? lo : (a > hi ? hi : a); }

// ------------------------------------------------------- ghost (clamp) fill
// 2D kernels of radius <= 4 (one-vector x frame) keep this loop form of the
// frame fill: the per-thread plans below measured 3-7 % slower there (code
// layout of the unrolled body), while they are 9-22 % faster in 3D.
// Tasks that overwrite the out-of-grid frame (width 4 in x) of a padded plane
// with clamped border values, in groups of four cells.
struct GhostX4 {
    int ntask, nA, nc;      // total tasks, column tasks, columns per in-grid row (0..2)
    int rA0;                // first in-grid padded row
    int cL, cR;             // padded float4 columns at x = -4 and x = nx (or -1)
    int srcL, srcR;         // padded x of global x = 0 and x = nx-1
    int rT0, nT, srcT;      // top ghost rows, their count, padded source row
    int rB0, nB, srcB;      // bottom ghost rows
    int cg0, ncg;           // float4 columns of the ghost rows
};

__device__ __forceinline__ GhostX4 make_ghost_x4(int ox, int oy, int pw, int ph, int nx, int nyp, int r)
{
    GhostX4 g;
    const int xL = -4 - ox, xR = nx - ox;
    g.cL = (xL >= 0 && xL + 4 <= pw) ? xL / 4 : -1;
    g.cR = (xR >= 0 && xR + 4 <= pw) ? xR / 4 : -1;
    g.srcL = -ox;
    g.srcR = nx - 1 - ox;
    g.nc = (g.cL >= 0) + (g.cR >= 0);
    const int a0 = max(0, oy), a1 = min(nyp, oy + ph);
    g.rA0 = a0 - oy;
    g.nA = (a1 > a0 ? a1 - a0 : 0) * g.nc;
    const int t0 = max(-r, oy), t1 = min(0, oy + ph);
    g.rT0 = t0 - oy;
    g.nT = t1 > t0 ? t1 - t0 : 0;
    g.srcT = -oy;
    const int b0 = max(nyp, oy), b1 = min(nyp + r, oy + ph);
    g.rB0 = b0 - oy;
    g.nB = b1 > b0 ? b1 - b0 : 0;
    g.srcB = nyp - 1 - oy;
    const int x0 = max(-4, ox), x1 = min(nx + 4, ox + pw);
    g.cg0 = (x0 - ox) / 4;
    g.ncg = x1 > x0 ? (x1 - x0) / 4 : 0;
    g.ntask = g.nA + (g.nT + g.nB) * g.ncg;
    return g;
}

// Cells are moved as raw bits, four at a time: 4-byte cells (FP32 rings, FP32
// input) or 2-byte cells (BF16/FP16 input).
template <int ES>
__device__ __forceinline__ void ghost_fill_x4(void *plane_, const GhostX4 &g, int pw, int ox, int nx, int tid, int nthr)
{
    using W = typename std::conditional<ES == 4, uint32_t, uint16_t>::type;
    using V = typename std::conditional<ES == 4, uint4, uint2>::type;
    W *plane = static_cast<W *>(plane_);
    auto bcast = [](W e) -> V {
        if constexpr (ES == 4) {
            return make_uint4(e, e, e, e);
        } else {
            const uint32_t u = static_cast<uint32_t>(e) | (static_cast<uint32_t>(e) << 16);
            return make_uint2(u, u);
        }
    };
    for (int t = tid; t < g.ntask; t += nthr) {
        int row, col;
        V v;
        if (t < g.nA) {
            row = g.rA0 + t / g.nc;
            const bool left = (t % g.nc == 0) && g.cL >= 0;
            col = left ? g.cL : g.cR;
            v = bcast(plane[row * pw + (left ? g.srcL : g.srcR)]);
        } else {
            const int u = t - g.nA;
            const int gr = u / g.ncg;
            col = g.cg0 + u % g.ncg;
            int srow;
            if (gr < g.nT) { row = g.rT0 + gr; srow = g.srcT; }
            else { row = g.rB0 + gr - g.nT; srow = g.srcB; }
            const int x4 = ox + 4 * col;
            if (x4 < 0) v = bcast(plane[srow * pw + g.srcL]);
            else if (x4 >= nx) v = bcast(plane[srow * pw + g.srcR]);
            else v = *reinterpret_cast<const V *>(plane + srow * pw + 4 * col);
        }
        *reinterpret_cast<V *>(plane + row * pw + 4 * col) = v;
    }
}

// Tasks that overwrite the out-of-grid frame (fw = 4*nv cells in x, r rows in
// y) of a padded plane with clamped border values, in groups of four cells.
struct Ghost {
    int ntask, nA, nc;      // total tasks, column tasks, frame columns per in-grid row
    int rA0;                // first in-grid padded row
    int cL0, nL, cR0;       // left frame: nL 4-cell columns from cL0; right frame from cR0
    int srcL, srcR;         // padded x of global x = 0 and x = nx-1
    int rT0, nT, srcT;      // top ghost rows, their count, padded source row
    int rB0, nB, srcB;      // bottom ghost rows
    int cg0, ncg;           // 4-cell columns of the ghost rows
};

__device__ __forceinline__ Ghost make_ghost(int ox, int oy, int pw, int ph, int nx, int nyp, int r, int fw)
{
    Ghost g;
    // left frame x in [-fw, 0), right frame x in [nx, nx + fw), clipped to the plane
    const int l0 = max(-fw - ox, 0), l1 = min(-ox, pw);
    const int q0 = max(nx - ox, 0), q1 = min(nx + fw - ox, pw);
    g.cL0 = l0 / 4;
    g.nL = l1 > l0 ? (l1 - l0) / 4 : 0;
    g.cR0 = q0 / 4;
    const int nR = q1 > q0 ? (q1 - q0) / 4 : 0;
    g.srcL = -ox;
    g.srcR = nx - 1 - ox;
    g.nc = g.nL + nR;
    const int a0 = max(0, oy), a1 = min(nyp, oy + ph);
    g.rA0 = a0 - oy;
    g.nA = (a1 > a0 ? a1 - a0 : 0) * g.nc;
    const int t0 = max(-r, oy), t1 = min(0, oy + ph);
    g.rT0 = t0 - oy;
    g.nT = t1 > t0 ? t1 - t0 : 0;
    g.srcT = -oy;
    const int b0 = max(nyp, oy), b1 = min(nyp + r, oy + ph);
    g.rB0 = b0 - oy;
    g.nB = b1 > b0 ? b1 - b0 : 0;
    g.srcB = nyp - 1 - oy;
    const int x0 = max(-fw, ox), x1 = min(nx + fw, ox + pw);
    g.cg0 = (x0 - ox) / 4;
    g.ncg = x1 > x0 ? (x1 - x0) / 4 : 0;
    g.ntask = g.nA + (g.nT + g.nB) * g.ncg;
    return g;
}

// Each thread's share of the frame tasks, resolved once per tile: task j moves
// four cells to cell offset dst[j] (< 0: none), from offset src[j] (four cells)
// or, for src[j] < 0, the single cell -src[j]-1 broadcast (clamp).
template <int MAXT> struct GhostPlan {
    int dst[MAXT], src[MAXT];
};

template <int MAXT>
__device__ __forceinline__ GhostPlan<MAXT> plan_ghost(const Ghost &g, int pw, int ox, int nx, int tid, int nthr,
                                                      int plane_cells = 0, unsigned *status = nullptr)
{
    GhostPlan<MAXT> p;
#pragma unroll
    for (int j = 0; j < MAXT; ++j) {
        const int t = tid + j * nthr;
        p.dst[j] = -1;
        p.src[j] = 0;
        if (t >= g.ntask) continue;
        int row, col, src;
        if (t < g.nA) {
            row = g.rA0 + t / g.nc;
            const int c = t % g.nc;
            const bool left = c < g.nL;
            col = left ? g.cL0 + c : g.cR0 + (c - g.nL);
            src = -(row * pw + (left ? g.srcL : g.srcR)) - 1;
        } else {
            const int u = t - g.nA;
            const int gr = u / g.ncg;
            col = g.cg0 + u % g.ncg;
            int srow;
            if (gr < g.nT) { row = g.rT0 + gr; srow = g.srcT; }
            else { row = g.rB0 + gr - g.nT; srow = g.srcB; }
            const int x4 = ox + 4 * col;
            if (x4 < 0) src = -(srow * pw + g.srcL) - 1;
            else if (x4 >= nx) src = -(srow * pw + g.srcR) - 1;
            else src = srow * pw + 4 * col;
        }
        p.dst[j] = row * pw + 4 * col;
        p.src[j] = src;
        if (status) {   // checked build: every task must stay inside the plane
            const int s0 = src < 0 ? -src - 1 : src;
            if (p.dst[j] < 0 || p.dst[j] + 4 > plane_cells || s0 < 0 || s0 + (src < 0 ? 1 : 4) > plane_cells) {
                atomicOr(status, kStatusBounds);
                p.dst[j] = -1;
            }
        }
    }
    return p;
}

// Cells are moved as raw bits: 4-byte cells (FP32 rings, FP32 input) or 2-byte
// cells (BF16/FP16 input).  Branch-free: a broadcast reads the same cell four
// times (stride 0), a copy four neighbouring cells (stride 1).
template <int ES, int MAXT>
__device__ __forceinline__ void ghost_apply(void *plane_, const GhostPlan<MAXT> &p)
{
    using W = typename std::conditional<ES == 4, uint32_t, uint16_t>::type;
    W *plane = static_cast<W *>(plane_);
#pragma unroll
    for (int j = 0; j < MAXT; ++j) {
        if (p.dst[j] < 0) continue;
        const int bc = p.src[j] < 0;
        const W *sp = plane + (bc ? -p.src[j] - 1 : p.src[j]);
        const int st = bc ? 0 : 1;
        W e[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) e[c] = sp[c * st];
        if constexpr (ES == 4) {
            *reinterpret_cast<uint4 *>(plane + p.dst[j]) = make_uint4(e[0], e[1], e[2], e[3]);
        } else {
            *reinterpret_cast<uint2 *>(plane + p.dst[j]) =
                make_uint2(static_cast<uint32_t>(e[0]) | (static_cast<uint32_t>(e[1]) << 16),
                           static_cast<uint32_t>(e[2]) | (static_cast<uint32_t>(e[3]) << 16));
        }
    }
}

__device__ __forceinline__ void mbar_inval(uint32_t bar)
{
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(bar) : "memory");
}

// ------------------------------------------------------------------ one tile
// Planes [Z0, Z1) of tile column `col` = tile_x + ntx * tile_y of one pass, by
// one thread block.  Returns false if a bounded wait expired (the device
// status word is then set).  Leaves the block's shared memory free for the
// next piece.
template <int D, int R, int T, int VY, typename S, int TX, int TY, bool SH, bool CHK, int P>
__device__ __forceinline__ bool sweep_tile(const CUtensorMap *tmap, const SweepArgs &a, int col, int Z0, int Z1,
                                           unsigned char *smem)
{
    using G = Geo<D, R, T, VY, static_cast<int>(sizeof(S)), TX, TY, P>;
    static_assert(D == 2 || D == 3, "dim");
    static_assert(R >= 1 && R <= kMaxR, "radius");
    static_assert(D == 3 || (VY == 1 && TY == 1), "2D keeps one row per thread");
    static_assert(G::OK, "tile too small for this temporal degree");
    constexpr int QP = G::QP;
    constexpr int U = G::U, NQ = G::NQ;
    constexpr bool ROT = G::ROT;
    constexpr bool WRAP = G::WRAP;   // input ring wraps inside a chunk (3D radius 1, P = 1)
    static_assert(!WRAP || P == 1, "wrapping ring: one plane per step");
    constexpr bool F32S = G::F32S;
    constexpr int PADIN = G::PADIN;
    constexpr int K2 = 2 * D;
    constexpr int PW = G::PW, PWIN = G::PWIN;
    constexpr int NTHR = TX * TY;
    constexpr int DEPTH = G::DEPTH, DS = G::DS;
    constexpr int SLOT32 = G::SLOT32, SLOTIN = G::SLOTIN;

    uint64_t *bars = reinterpret_cast<uint64_t *>(smem);
    volatile int *sflag = reinterpret_cast<volatile int *>(smem + 8 * kMaxDepthIn);
    S *ring_in = reinterpret_cast<S *>(smem + kSmemHeader);
    float *rings = reinterpret_cast<float *>(smem + kSmemHeader + DEPTH * SLOTIN * sizeof(S));
    // FP32 ring of level s (1..T-1), slot j = plane mod QP; level 0 is the input ring
    auto ring32 = [&](int s, int j) -> float * { return rings + ((s - 1) * QP + j) * SLOT32; };

    const int tx = threadIdx.x, ty = threadIdx.y;
    const int tid = ty * TX + tx;
    // CHK (bounds-checked instantiations, a substitute for a memory checker): every
    // shared-memory access must fall in the block's rings, every global store in the
    // output grid, every copy inside its slot and the grid; a violation sets
    // kStatusBounds in the device status and the access is skipped.
    auto smem_ok = [&](const void *ptr, int bytes) -> bool {
        if constexpr (!CHK) {
            (void)ptr;
            (void)bytes;
            return true;
        } else {
            const unsigned char *q = static_cast<const unsigned char *>(ptr);
            const bool ok = q >= smem + kSmemHeader && q + bytes <= smem + G::SMEM;
            if (!ok) atomicOr(a.status, kStatusBounds);
            return ok;
        }
    };

    // 2D: the coefficients live in per-thread registers (the empty asm hides that they
    // are uniform), so each FMA reads them from the register file instead of uniform
    // registers refilled from the constant bank inside the loop (measured 2-8 % faster
    // for r >= 2; 3D kernels, tighter on registers, gain nothing and keep the default).
    // SH: one coefficient per distance, c[0] centre and c[i] for distance i.
    constexpr int K = SH ? 1 + R : 1 + 2 * D * R;
    // Packed two-lane FP32 arithmetic (cells 0,1 and 2,3 of a row in lockstep; bit-identical
    // to the scalar chain) where it measured faster: 3D FP32 one-level passes of radius 3
    // (+3 %, coefficient pairs read from the kernel parameters) and 4 (+1.3 %, pairs held in
    // registers).  Elsewhere its 30-40 extra registers cost more than the issue slots it saves.
    constexpr bool PK = !SH && D == 3 && T == 1 && F32S && (R == 3 || R == 4);
    constexpr bool PKC = R == 3;   // coefficient pairs from the parameters (else registers)
    auto cpair = [&](int k) -> uint64_t {   // coefficient k in both lanes
        if constexpr (PKC) return *reinterpret_cast<const uint64_t *>(&a.cc[2 * k]);
        else return 0;
    };
    float cf[K];
#pragma unroll
    for (int i = 0; i < K; ++i) {
        cf[i] = a.c[i];
        if constexpr (D == 2) asm volatile("" : "+f"(cf[i]));
    }

    // ---- tile of this piece
    const int tile_x = col % a.ntx;
    const int tile_y = (D == 3) ? col / a.ntx : 0;
    const int gx0 = tile_x * G::CX - G::HTX;          // thread-region origin
    const int gy0 = (D == 3) ? tile_y * G::CY - G::HTY : 0;
    const int ox = gx0 - G::PAD32;                     // padded FP32 plane origin
    const int oy = (D == 3) ? gy0 - R : 0;
    const int ox_in = gx0 - PADIN;                     // padded input plane origin
    const int last = a.ns - 1;

    // ---- this thread's cells
    const int xl = 4 * tx;
    const int yl0 = ty * VY;
    const int prow0 = (D == 3) ? yl0 + R : 0;          // padded row of own row 0
    const int toff = prow0 * PW + xl + G::PAD32;       // own cell 0 in an FP32 plane
    const int toffin = prow0 * PWIN + xl + PADIN;      // own cell 0 in an input plane
    const int gx = gx0 + xl;
    const bool xstore = xl >= G::HTX && xl < G::HTX + G::CX && gx < a.nx;
    // radius 1: x neighbours by shuffles within the lanes of one x row (a warp in 2D, 16 lanes
    // of one thread row in 3D) except on these lanes (row segment ends, grid edges).  3D
    // passes of one level keep the shared-memory loads (measured 6 % faster on 512^3; two or
    // three levels run 3-8 % faster with shuffles).
    constexpr bool SHX = R == 1 && (D == 2 || (TX == 16 && T >= 2));
    constexpr int SW = TX < 32 ? TX : 32;              // shuffle segment width
    const bool xedge = (tx % SW) == 0 || (tx % SW) == SW - 1 || gx <= 0 || gx + 4 >= a.nx;
    (void)xedge;
    bool ystore[VY];
#pragma unroll
    for (int vy = 0; vy < VY; ++vy) {
        const int yl = yl0 + vy;
        ystore[vy] = (D == 2) || (yl >= G::HTY && yl < G::HTY + G::CY && gy0 + yl < a.ny);
    }
    const int64_t pstride = (D == 3) ? static_cast<int64_t>(a.nx) * a.ny : a.nx;
    S *const gout = static_cast<S *>(a.out) +
                    ((D == 3) ? static_cast<int64_t>(gy0 + yl0) * a.nx : 0) + gx;

    // A thread whose VY rows cross the grid's top or bottom edge keeps its
    // out-of-grid rows equal to the border row in registers (clamp), since
    // its in-grid rows take y neighbours from its own registers.
    const int vz = -(gy0 + yl0);                       // own row index of global y = 0
    const int vb = a.ny - 1 - (gy0 + yl0);             // own row index of global y = ny-1
    const bool top_cross = (D == 3) && VY > 1 && vz > 0 && vz < VY;
    const bool bot_cross = (D == 3) && VY > 1 && vb >= 0 && vb < VY - 1;
    // block-uniform: the thread region reaches past the grid's top or bottom edge (only such
    // tiles have threads whose rows cross it).  Radius 1 and 4 skip the clamp in other tiles
    // with a branch (+2 % and +1 % on 512^3 against the branch-free selects); radius 2
    // and 3 keep the selects (the branch splits the step's straight-line code: -5 % at r = 3).
    constexpr bool YBR = R == 1 || R == 4;
    const bool ytile = (D == 3) && VY > 1 && (!YBR || gy0 < 0 || gy0 + G::BY > a.ny);
    auto clamp_rows = [&](float (&v)[VY][4]) {
        if (top_cross) {
#pragma unroll
            for (int vy = VY - 2; vy >= 0; --vy)
                if (vy < vz)
#pragma unroll
                    for (int c = 0; c < 4; ++c) v[vy][c] = v[vy + 1][c];
        }
        if (bot_cross) {
#pragma unroll
            for (int vy = 1; vy < VY; ++vy)
                if (vy > vb)
#pragma unroll
                    for (int c = 0; c < 4; ++c) v[vy][c] = v[vy - 1][c];
        }
    };

    // ---- plane ranges: level s covers planes [lo[s], hi[s]]; step k handles its planes
    // P*k - lag(s) + j, j < P
    auto fdiv = [](int a, int b) { return a >= 0 ? a / b : -((-a + b - 1) / b); };
    int lo[T + 1], hi[T + 1];
    int kA = 0, kB = 0x7fffffff;
#pragma unroll
    for (int s = 0; s <= T; ++s) {
        lo[s] = max(Z0 - (T - s) * R, 0);
        hi[s] = Z1 - 1 + (T - s) * R;
        kA = max(kA, cdiv(max(lo[s], 1) + G::lag(s), P));
        kB = min(kB, fdiv(min(hi[s], last) + G::lag(s) + 1 - P, P));
    }
    // steps in [kA, kB] have every plane of every level active, inside the grid and past plane 0
    const int k0 = lo[0] / P;                          // first step (level 0 loads plane lo[0])
    const int k1 = (Z1 - 1 + G::lag(T)) / P;           // last step (level T stores plane Z1 - 1)
    const int lmax = min(hi[0], last);                 // last input plane to load
    const int smax = lmax / P;                         // last step with an input plane to load
    const int lap0 = k0 / DS;

    // clamp frames (x: the 4*NV cells the neighbour loads reach; 3D y: r rows) of the
    // FP32 rings and of the input ring, each thread's tasks resolved once per tile
    constexpr int FW = 4 * G::NV;
    constexpr bool SAME = F32S && G::PADIN == G::PAD32;   // input ring laid out like the FP32 rings
    constexpr int MT32 = cdiv((D == 3) ? G::PH * 2 * G::NV + 2 * R * (PW / 4) : 2 * G::NV, NTHR);
    constexpr int MTIN = cdiv((D == 3) ? G::PH * 2 * G::NV + 2 * R * (PWIN / 4) : 2 * G::NV, NTHR);
    constexpr bool X4 = D == 2 && G::NV == 1 && !CHK;   // loop-form fill (GhostX4)
    const Ghost g32 = make_ghost(ox, oy, PW, G::PH, a.nx, (D == 3) ? a.ny : 1, R, FW);
    const bool gh_on = g32.ntask > 0;                  // block-uniform: tile touches an x or y edge
    GhostPlan<X4 ? 1 : MT32> gp32;
    GhostPlan<(X4 || SAME) ? 1 : MTIN> gpin;
    GhostX4 gx32, gxin;
    if constexpr (X4) {
        gx32 = make_ghost_x4(ox, oy, PW, G::PH, a.nx, 1, R);
        gxin = F32S ? gx32 : make_ghost_x4(ox_in, oy, PWIN, G::PH, a.nx, 1, R);
    } else {
        gp32 = plan_ghost<MT32>(g32, PW, ox, a.nx, tid, NTHR, PW * G::PH, CHK ? a.status : nullptr);
        if constexpr (!SAME) {
            const Ghost gin = make_ghost(ox_in, oy, PWIN, G::PH, a.nx, (D == 3) ? a.ny : 1, R, FW);
            gpin = plan_ghost<MTIN>(gin, PWIN, ox_in, a.nx, tid, NTHR, PWIN * G::PH, CHK ? a.status : nullptr);
        }
    }
    (void)gp32;
    (void)gpin;
    (void)gx32;
    (void)gxin;

    if (tid == 0) {
        for (int i = 0; i < DS; ++i) mbar_init(smem_addr(bars + i), 1);
        // step slots before k0's slot are first used one lap later: retire their phase 0 now
        for (int i = 0; i < k0 % DS; ++i) mbar_arrive(smem_addr(bars + i));
        *sflag = 0;
        fence_mbar_init();
    }
    __syncthreads();

    // One thread issues the input loads of a step: step kq brings planes P*kq + j (j < P, up
    // to lmax) into the P slots of step slot kq mod DS, completing one mbarrier phase.  Thread
    // 0 issues the prologue's loads, and every later step's too, except in 2D kernels with
    // 16-bit storage and several rows per step (RPROD): there the producer rotates over the
    // block's warps (lane 0 of warp k mod NW at step k), so that no warp carries the issue
    // work of every step into the step's barrier (measured +3 to +8 % for BF16/FP16 r = 2..4;
    // one-row kernels lost 3 %, 2D FP32 kernels gained nothing, and 3D ones need more
    // registers for it).  The producers' record of what was issued and waited for
    // (issued_hi, consumed_hi) serves the drain after an abort.
    constexpr bool RPROD = D == 2 && !F32S && P >= 2;
    constexpr int NW = NTHR / 32;
    static_assert(NW >= 1 && (NW & (NW - 1)) == 0, "whole warps, a power of two");
    int issued_hi = k0 - 1;
    auto issue = [&](int kq) {
        const int sslot = kq % DS;
        const uint32_t bar = smem_addr(bars + sslot);
        S *dst0 = ring_in + sslot * P * SLOTIN;
        if constexpr (!RPROD) issued_hi = kq;
        if (a.fault_plane >= P * kq && a.fault_plane < P * kq + P) return;   // test hook: never complete
        if constexpr (D == 2) {
            const int xa = max(ox_in, 0), xb = min(ox_in + PWIN, a.nx);
            uint32_t bytes = xb > xa ? static_cast<uint32_t>((xb - xa) * sizeof(S)) : 0u;
            const int nq = P == 1 ? 1 : min(P, lmax - P * kq + 1);   // planes of this step inside the grid
            if constexpr (CHK) {   // destination inside the slot, source inside the grid, 16-byte units
                const int64_t src = static_cast<int64_t>(P * kq) * a.nx + xa;
                const bool ok = xa - ox_in >= 0 && (xa - ox_in) * sizeof(S) + bytes <= SLOTIN * sizeof(S) &&
                                src >= 0 && (src + static_cast<int64_t>(nq - 1) * a.nx) * sizeof(S) + bytes <=
                                                static_cast<int64_t>(a.nx) * a.ns * sizeof(S) &&
                                bytes % 16 == 0 && (src * sizeof(S)) % 16 == 0 && ((xa - ox_in) * sizeof(S)) % 16 == 0;
                if (!ok) {
                    atomicOr(a.status, kStatusBounds);
                    bytes = 0;
                }
            }
            mbar_arrive_expect_tx(bar, bytes * static_cast<uint32_t>(nq));
            if (bytes) {
                const S *src = static_cast<const S *>(a.in) + static_cast<int64_t>(P * kq) * a.nx + xa;
#pragma unroll
                for (int j = 0; j < P; ++j)
                    if (j < nq) bulk_load(smem_addr(dst0 + j * SLOTIN + (xa - ox_in)), src + static_cast<int64_t>(j) * a.nx, bytes, bar);
            }
        } else {
            const int q = kq;   // 3D: one plane per step
            if constexpr (CHK) {   // the box's x coordinate must be 16-byte aligned
                if ((ox_in * static_cast<int>(sizeof(S))) % 16 != 0 || q < 0 || q >= a.ns) {
                    atomicOr(a.status, kStatusBounds);
                    mbar_arrive_expect_tx(bar, 0);
                    return;
                }
            }
            mbar_arrive_expect_tx(bar, static_cast<uint32_t>(PWIN * G::PH * sizeof(S)));
            tma_load_3d(smem_addr(dst0), tmap, ox_in, oy, q, bar);
        }
    };
    {
        const int qe = min(k0 + G::PFS - 1, smax);
        if (tid == 0)
            for (int kq = k0; kq <= qe; ++kq) issue(kq);
        if constexpr (RPROD) issued_hi = max(issued_hi, qe);   // every thread keeps the record
    }

    float q[T][NQ][VY][4];
#pragma unroll
    for (int s = 0; s < T; ++s)
#pragma unroll
        for (int j = 0; j < NQ; ++j)
#pragma unroll
            for (int vy = 0; vy < VY; ++vy)
#pragma unroll
                for (int v = 0; v < 4; ++v) q[s][j][vy][v] = 0.f;

    int consumed_hi = k0 - 1;   // last input step waited for
    bool aborted = false;

    // per-chunk state (a chunk is U steps; kb is a multiple of U)
    int kb = k0 - k0 % U;
    int kb_mod = kb % DS;       // step slot of step kb
    int lap = kb / DS;
    uint32_t bar0 = 0, par = 0;
    const uint32_t bars_a = smem_addr(bars);
    (void)bars_a;
    // WRAP: step slot of step kb + J (a chunk wraps past the ring's end at most once)
    auto wslot = [&](int J) { return kb_mod + J >= DS ? kb_mod + J - DS : kb_mod + J; };
    (void)wslot;
    const S *inb = nullptr;     // own cell 0 in the input slot of plane P*kb
    const S *inbp = nullptr;    // ROT: own cell 0 in the input slot of plane P*kb - QP
    S *inslot = nullptr;        // input slot of plane P*kb
    // shifting queue (P = 1): FP32 ring slot of plane kb - lag(s) for level s = 1..T
    int rb[T + 1];
#pragma unroll
    for (int s = 1; s <= T; ++s) rb[s] = cmod(kb - G::lag(s), QP);

    // queue index of plane P*k - lag(s) + j, which level s computes at chunk step J
    auto qnew = [](int s, int J, int j) constexpr { return ROT ? cmod(P * J - G::lag(s) + j, QP) : QP + J; };
    // queue index of level s-1's plane p+e, read by level s at chunk step J for its plane
    // p = P*k - lag(s) + j (|e| <= R); level s-1 has computed plane p+R in this step (s = 1)
    // or in an earlier one (s >= 2)
    auto qrd = [](int s, int J, int j, int e) constexpr {
        return ROT ? cmod(P * J - G::lag(s) + j + e, QP) : (s == 1 ? QP + J : QP + J - 1) - (R - e);
    };
    // FP32 ring slot of level s's plane P*(k - off) - lag(s) + j at chunk step J (off = 0 or 1)
    auto rslot = [&](int s, int J, int j, int off) -> int {
        if constexpr (ROT) {
            return cmod(P * (J - off) - G::lag(s) + j, QP);
        } else {
            int jj = rb[s] + J - off;
            jj = jj >= QP ? jj - QP : jj;
            return jj < 0 ? jj + QP : jj;
        }
    };

    // ---- plane j of time level s at step k
    auto level = [&](auto sc, auto Jc, auto jc, auto CKc, int k) {
        constexpr int s = decltype(sc)::value;
        constexpr int J = decltype(Jc)::value;
        constexpr int j = decltype(jc)::value;
        constexpr bool CK = decltype(CKc)::value;
        constexpr int jn = qnew(s, J, j);              // own queue index of plane p
        constexpr int jcq = qrd(s, J, j, 0);           // level s-1's queue index of plane p
        const int p = P * k - G::lag(s) + j;
        if constexpr (CK) {
            if (p < lo[s] || p > hi[s]) return;
            if (p > last) {   // beyond the end of the stream: repeat the last plane (clamp)
                if constexpr (s < T) {
#pragma unroll
                    for (int vy = 0; vy < VY; ++vy)
#pragma unroll
                        for (int v = 0; v < 4; ++v) q[s][jn][vy][v] = q[s][ROT ? cmod(jn - 1, QP) : jn - 1][vy][v];
                }
                return;
            }
        }
        // level s-1's plane p in shared memory at this thread's cell 0: level 1 reads the
        // input ring (storage type, widened exactly on load), higher levels the FP32 rings
        const S *own_in = nullptr;
        const float *own32 = nullptr;
        if constexpr (s == 1) {
            if constexpr (WRAP) {
                int d = wslot(J) - G::L1;               // input slot of plane k - L1
                d = d < 0 ? d + DS : d;
                own_in = ring_in + d * SLOTIN + toffin;
            } else if constexpr (ROT) {
                constexpr int d = P * J - G::L1 + j;    // input slot of plane p relative to plane P*kb
                own_in = d >= 0 ? inb + d * SLOTIN : inbp + (d + QP) * SLOTIN;
            } else {
                int d = kb_mod + J - R;     // input slot of plane k-R (P = 1)
                d = d < 0 ? d + DEPTH : d;
                own_in = ring_in + d * SLOTIN + toffin;
            }
        } else {
            own32 = ring32(s - 1, rslot(s, J, j, 0)) + toff;
        }
        auto ld = [&](int row, int dx, float (&v)[4]) {
            if constexpr (s == 1) {
                if (smem_ok(own_in + row * PWIN + dx, 4 * sizeof(S))) Fmt<S>::load4(own_in + row * PWIN + dx, v);
                else v[0] = v[1] = v[2] = v[3] = 0.f;
            } else {
                if (smem_ok(own32 + row * PW + dx, 16)) Fmt<float>::load4(own32 + row * PW + dx, v);
                else v[0] = v[1] = v[2] = v[3] = 0.f;
            }
        };
        float up[(D == 3) ? R : 1][4], dn[(D == 3) ? R : 1][4];
        (void)up;
        (void)dn;
        if constexpr (D == 3) {
#pragma unroll
            for (int m = 0; m < R; ++m) {
                ld(-(m + 1), 0, up[m]);
                ld(VY + m, 0, dn[m]);
            }
        }
        constexpr int NV = G::NV;
        float res[VY][4];
        uint64_t cpr[PK && !PKC ? K : 1];   // coefficient pairs held in registers
        (void)cpr;
        if constexpr (PK && !PKC) {
#pragma unroll
            for (int i = 0; i < K; ++i) cpr[i] = pk2(cf[i], cf[i]);
        }
        auto cp = [&](int k) -> uint64_t {
            if constexpr (PK && !PKC) return cpr[k];
            else return cpair(k);
        };
        (void)cp;
#pragma unroll
        for (int vy = 0; vy < VY; ++vy) {
            // L[m] holds cells x0-4(m+1) .. x0-4m-1, Rr[m] cells x0+4(m+1) .. x0+4m+7
            float L[NV][4], Rr[NV][4];
            if constexpr (SHX) {
                // radius 1 needs one cell on each side: the neighbouring lanes' own cells
                // of the same plane; warp-edge and grid-edge lanes read shared memory
                // (the neighbouring warp's cells, or the clamp frame)
                const float(&c0)[VY][4] = q[s - 1][jcq];
                float l3 = __shfl_up_sync(0xffffffffu, c0[vy][3], 1, SW);
                float r0 = __shfl_down_sync(0xffffffffu, c0[vy][0], 1, SW);
                if (xedge) {
                    float t4[4];
                    ld(vy, -4, t4);
                    l3 = t4[3];
                    ld(vy, 4, t4);
                    r0 = t4[0];
                }
#pragma unroll
                for (int v = 0; v < 4; ++v) L[0][v] = Rr[0][v] = 0.f;
                L[0][3] = l3;
                Rr[0][0] = r0;
            } else {
#pragma unroll
                for (int m = 0; m < NV; ++m) {
                    ld(vy, -4 * (m + 1), L[m]);
                    ld(vy, 4 * (m + 1), Rr[m]);
                }
            }
            const float(&ctr)[VY][4] = q[s - 1][jcq];
            if constexpr (PK) {
                // cell v + d of this row (|d| <= 4*NV): own vector, or the left/right neighbour vectors
                auto nb = [&](int v, int d) -> float {
                    const int x = v + d;
                    if (x >= 0 && x <= 3) return ctr[vy][cclamp(x, 0, 3)];
                    if (x < 0) return L[cclamp((-x - 1) / 4, 0, NV - 1)][cclamp(x + 4 * ((-x - 1) / 4 + 1), 0, 3)];
                    return Rr[cclamp(x / 4 - 1, 0, NV - 1)][cclamp(x % 4, 0, 3)];
                };
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int v = 2 * h;   // cells v and v + 1 in the two lanes
                    uint64_t acc = mul2(cp(0), pk2(ctr[vy][v], ctr[vy][v + 1]));
#pragma unroll
                    for (int i = 1; i <= R; ++i) {
                        const int cb = 1 + (i - 1) * K2;
                        if ((i & 1) == 0) {   // even distance: both x neighbours are register pairs too
                            acc = fma2(cp(cb + 0), pk2(nb(v, -i), nb(v + 1, -i)), acc);
                            acc = fma2(cp(cb + 1), pk2(nb(v, i), nb(v + 1, i)), acc);
                        } else {              // odd distance: one lane at a time
                            float a0, a1;
                            upk2(acc, a0, a1);
                            a0 = __fmaf_rn(cf[cb + 0], nb(v, -i), a0);
                            a1 = __fmaf_rn(cf[cb + 0], nb(v + 1, -i), a1);
                            a0 = __fmaf_rn(cf[cb + 1], nb(v, i), a0);
                            a1 = __fmaf_rn(cf[cb + 1], nb(v + 1, i), a1);
                            acc = pk2(a0, a1);
                        }
                        if constexpr (D == 3) {
                            const float *sp = (vy - i >= 0) ? &ctr[cclamp(vy - i, 0, VY - 1)][0] : &up[cclamp(i - vy - 1, 0, R - 1)][0];
                            const float *np = (vy + i < VY) ? &ctr[cclamp(vy + i, 0, VY - 1)][0] : &dn[cclamp(vy + i - VY, 0, R - 1)][0];
                            acc = fma2(cp(cb + 2), pk2(sp[v], sp[v + 1]), acc);
                            acc = fma2(cp(cb + 3), pk2(np[v], np[v + 1]), acc);
                        }
                        const float(&bq)[VY][4] = q[s - 1][qrd(s, J, j, -i)];
                        const float(&aq)[VY][4] = q[s - 1][qrd(s, J, j, i)];
                        acc = fma2(cp(cb + K2 - 2), pk2(bq[vy][v], bq[vy][v + 1]), acc);
                        acc = fma2(cp(cb + K2 - 1), pk2(aq[vy][v], aq[vy][v + 1]), acc);
                    }
                    upk2(acc, res[vy][v], res[vy][v + 1]);
                }
                continue;
            }
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                float acc = __fmul_rn(cf[0], ctr[vy][v]);
#pragma unroll
                for (int i = 1; i <= R; ++i) {
                    const int cb = SH ? i : 1 + (i - 1) * K2;
                    const float w = (v - i >= 0) ? ctr[vy][cclamp(v - i, 0, 3)]
                                                 : L[cclamp((i - v - 1) / 4, 0, NV - 1)][cclamp(v - i + 4 * ((i - v - 1) / 4 + 1), 0, 3)];
                    const float e = (v + i <= 3) ? ctr[vy][cclamp(v + i, 0, 3)]
                                                 : Rr[cclamp((v + i) / 4 - 1, 0, NV - 1)][cclamp((v + i) % 4, 0, 3)];
                    float sv = 0.f, nv = 0.f;
                    if constexpr (D == 3) {
                        sv = (vy - i >= 0) ? ctr[cclamp(vy - i, 0, VY - 1)][v] : up[cclamp(i - vy - 1, 0, R - 1)][v];
                        nv = (vy + i < VY) ? ctr[cclamp(vy + i, 0, VY - 1)][v] : dn[cclamp(vy + i - VY, 0, R - 1)][v];
                    }
                    const float bz = q[s - 1][qrd(s, J, j, -i)][vy][v];   // stream axis: S (2D) / B (3D)
                    const float az = q[s - 1][qrd(s, J, j, i)][vy][v];    // N (2D) / A (3D)
                    if constexpr (SH) {
                        // neighbours at distance i summed left to right (W, E, S, N[, B, A]),
                        // then one FMA with the shared coefficient
                        float sum = __fadd_rn(w, e);
                        if constexpr (D == 3) {
                            sum = __fadd_rn(sum, sv);
                            sum = __fadd_rn(sum, nv);
                        }
                        sum = __fadd_rn(sum, bz);
                        sum = __fadd_rn(sum, az);
                        acc = __fmaf_rn(cf[cb], sum, acc);
                    } else {
                        acc = __fmaf_rn(cf[cb + 0], w, acc);
                        acc = __fmaf_rn(cf[cb + 1], e, acc);
                        if constexpr (D == 3) {
                            acc = __fmaf_rn(cf[cb + 2], sv, acc);
                            acc = __fmaf_rn(cf[cb + 3], nv, acc);
                        }
                        acc = __fmaf_rn(cf[cb + K2 - 2], bz, acc);
                        acc = __fmaf_rn(cf[cb + K2 - 1], az, acc);
                    }
                }
                res[vy][v] = acc;
            }
        }
        // the last level's out-of-grid rows are neither stored nor read
        if constexpr (D == 3 && VY > 1 && s < T) {
            if (ytile) clamp_rows(res);
        }
        if constexpr (s == T) {
            if (xstore) {
                S *o = gout + static_cast<int64_t>(p) * pstride;
#pragma unroll
                for (int vy = 0; vy < VY; ++vy)
                    if (ystore[vy]) {
                        if constexpr (CHK) {   // inside the output grid, four whole cells of one row
                            const int64_t e = (o + vy * a.nx) - static_cast<S *>(a.out);
                            const int64_t total = static_cast<int64_t>(a.nx) * a.ny * a.nz;
                            if (e < 0 || e + 4 > total || gx + 4 > a.nx) {
                                atomicOr(a.status, kStatusBounds);
                                continue;
                            }
                        }
                        Fmt<S>::store4(o + vy * a.nx, res[vy]);
                    }
            }
        } else {
            float *dst = ring32(s, rslot(s, J, j, 0)) + toff;
#pragma unroll
            for (int vy = 0; vy < VY; ++vy) {
                if (smem_ok(dst + vy * PW, 16)) Fmt<float>::store4(dst + vy * PW, res[vy]);
#pragma unroll
                for (int v = 0; v < 4; ++v) q[s][jn][vy][v] = res[vy][v];
            }
            if constexpr (CK) {
                if (p == 0) {   // top clamp: planes -r..-1 of this level equal plane 0
#pragma unroll
                    for (int jj = 0; jj < NQ; ++jj)
#pragma unroll
                        for (int vy = 0; vy < VY; ++vy)
#pragma unroll
                            for (int v = 0; v < 4; ++v) q[s][jj][vy][v] = res[vy][v];
                }
            }
        }
    };

    // ---- level 0 of step k: take planes P*k + j from the input ring
    auto level0 = [&](auto Jc, auto CKc, int k) {
        constexpr int J = decltype(Jc)::value;
        constexpr bool CK = decltype(CKc)::value;
        if constexpr (CK) {
            if (P * k + P - 1 < lo[0] || P * k > hi[0]) return;
        }
        // the step's planes inside the grid were loaded together: one wait
        if (!CK || P * k <= last) {
            const bool ok = WRAP ? mbar_wait_bounded(bars_a + 8 * wslot(J), par ^ static_cast<uint32_t>(kb_mod + J >= DS),
                                                     a.timeout_ms)
                                 : mbar_wait_bounded(bar0 + 8 * J, par, a.timeout_ms);
            if (!ok) {
                *sflag = 1;
                atomicOr(a.status, kStatusTimeout);
                return;
            }
            if (RPROD || tid == 0) consumed_hi = k;
        }
        SFor<0, P>::run([&](auto jc) {
            constexpr int j = decltype(jc)::value;
            constexpr int jn = qnew(0, J, j);
            const int p = P * k + j;
            if constexpr (CK) {
                if (p < lo[0] || p > hi[0]) return;
                if (p > last) {
#pragma unroll
                    for (int vy = 0; vy < VY; ++vy)
#pragma unroll
                        for (int v = 0; v < 4; ++v) q[0][jn][vy][v] = q[0][ROT ? cmod(jn - 1, QP) : QP + J - 1][vy][v];
                    return;
                }
            }
            S *const slot = WRAP ? ring_in + wslot(J) * SLOTIN : inslot + (P * J + j) * SLOTIN;
            const S *src = slot + toffin;
            float v4[VY][4];
#pragma unroll
            for (int vy = 0; vy < VY; ++vy) {
                if (smem_ok(src + vy * PWIN, 4 * sizeof(S))) Fmt<S>::load4(src + vy * PWIN, v4[vy]);
                else v4[vy][0] = v4[vy][1] = v4[vy][2] = v4[vy][3] = 0.f;
            }
            if constexpr (D == 3 && VY > 1) {
                if (ytile) clamp_rows(v4);
            }
#pragma unroll
            for (int vy = 0; vy < VY; ++vy)
#pragma unroll
                for (int v = 0; v < 4; ++v) q[0][jn][vy][v] = v4[vy][v];
            if constexpr (CK) {
                if (p == 0) {
#pragma unroll
                    for (int jj = 0; jj < NQ; ++jj)
#pragma unroll
                        for (int vy = 0; vy < VY; ++vy)
#pragma unroll
                            for (int v = 0; v < 4; ++v) q[0][jj][vy][v] = v4[vy][v];
                }
            }
            // the input slot is level 0's ring: clamp its out-of-grid frame now (read from the
            // next step on)
            if (gh_on) {
                if constexpr (X4) ghost_fill_x4<sizeof(S)>(slot, gxin, PWIN, ox_in, a.nx, tid, NTHR);
                else if constexpr (SAME) ghost_apply<sizeof(S)>(slot, gp32);
                else ghost_apply<sizeof(S)>(slot, gpin);
            }
        });
    };

    // ---- one step
    auto step = [&](auto Jc, auto CKc) {
        constexpr int J = decltype(Jc)::value;
        constexpr bool CK = decltype(CKc)::value;
        const int k = kb + J;
        if (aborted) return;
        if constexpr (CK) {
            if (k < k0 || k > k1) return;
        }
        // keep PFS steps of input in flight
        {
            const int kn = k + G::PFS;
            if (kn <= smax) {
                if (tid == (RPROD ? (k & (NW - 1)) << 5 : 0)) {
                    if (gh_on) fence_proxy_async_smem();
                    issue(kn);
                }
                if constexpr (RPROD) issued_hi = kn;
            }
        }
        // levels T..2 highest first, then level 0 (the input), then level 1 (reads the input ring)
        SFor<0, T - 1>::run([&](auto ic) {
            constexpr int s = T - decltype(ic)::value;
            SFor<0, P>::run([&](auto jc) { level(IC<s>{}, Jc, jc, CKc, k); });
        });
        level0(Jc, CKc, k);
        SFor<0, P>::run([&](auto jc) { level(IC<1>{}, Jc, jc, CKc, k); });
        // clamp frame of ring planes written in the previous step
        if (gh_on) {
            SFor<1, T>::run([&](auto sc) {
                constexpr int s = decltype(sc)::value;
                SFor<0, P>::run([&](auto jc) {
                    constexpr int j = decltype(jc)::value;
                    const int p = P * (k - 1) - G::lag(s) + j;
                    if (p >= lo[s] && p <= min(hi[s], last)) {
                        if constexpr (X4) ghost_fill_x4<4>(ring32(s, rslot(s, J, j, 1)), gx32, PW, ox, a.nx, tid, NTHR);
                        else ghost_apply<4>(ring32(s, rslot(s, J, j, 1)), gp32);
                    }
                });
            });
        }
        __syncthreads();
        aborted = (*sflag != 0);
    };

    for (; kb <= k1 && !aborted; kb += U) {
        par = static_cast<uint32_t>((lap - lap0) & 1);
        bar0 = smem_addr(bars + kb_mod);
        inslot = ring_in + kb_mod * P * SLOTIN;
        inb = inslot + toffin;
        if constexpr (ROT && !WRAP) inbp = ring_in + (kb_mod == 0 ? DEPTH - QP : P * kb_mod - QP) * SLOTIN + toffin;
        if (kb >= kA && kb + U - 1 <= kB) {
            SFor<0, U>::run([&](auto Jc) { step(Jc, std::false_type{}); });
        } else {
            SFor<0, U>::run([&](auto Jc) { step(Jc, std::true_type{}); });
        }
        if constexpr (!ROT) {
            // shift every queue down by the U planes appended in this chunk
#pragma unroll
            for (int s = 0; s < T; ++s)
#pragma unroll
                for (int jj = 0; jj < QP; ++jj)
#pragma unroll
                    for (int vy = 0; vy < VY; ++vy)
#pragma unroll
                        for (int v = 0; v < 4; ++v) q[s][jj][vy][v] = q[s][jj + U][vy][v];
#pragma unroll
            for (int s = 1; s <= T; ++s) rb[s] = rb[s] + U >= QP ? rb[s] + U - QP : rb[s] + U;
        }
        kb_mod += U;
        if (kb_mod >= DS) {
            kb_mod -= DS;
            ++lap;
        }
    }

    if (aborted && tid == 0) {
        // let the copies still in flight land before the block's shared memory is released
        for (int kq = consumed_hi + 1; kq <= issued_hi; ++kq) {
            if (a.fault_plane >= P * kq && a.fault_plane < P * kq + P) continue;
            mbar_wait_bounded(smem_addr(bars + kq % DS), static_cast<uint32_t>((kq / DS - lap0) & 1), a.timeout_ms);
        }
    }
    __syncthreads();
    if (tid == 0)
        for (int i = 0; i < DS; ++i) mbar_inval(smem_addr(bars + i));
    __syncthreads();
    return !aborted;
}

// Work of block b.  flat: planes [b*seg, (b+1)*seg) of the tile columns laid
// end to end (column c holds planes c*ns .. c*ns + ns - 1), a range that
// crosses the end of a column being swept as one piece per column.  Slabs:
// column b mod (ntx*nty), planes [j*seg, (j+1)*seg) with j = b / (ntx*nty),
// so blocks running together cover neighbouring tiles of the same planes and
// share their overlapping halo reads in L2.
template <int D, int R, int T, int VY, typename S, int TX, int TY, bool SH, bool CHK, int P>
__device__ __forceinline__ bool sweep_block(const CUtensorMap *tmap, const SweepArgs &a, int b, unsigned char *smem)
{
    const int cols = a.ntx * a.nty;
    int64_t w, we;
    if (a.flat) {
        w = static_cast<int64_t>(b) * a.seg;
        we = min(w + a.seg, static_cast<int64_t>(cols) * a.ns);
    } else {   // slab j = b / cols of column b mod cols
        const int col = b % cols;
        const int z0 = (b / cols) * a.seg;
        w = static_cast<int64_t>(col) * a.ns + z0;
        we = static_cast<int64_t>(col) * a.ns + min(z0 + a.seg, a.ns);
    }
    bool ok = true;
    while (ok && w < we) {   // one sweep_tile call site: the kernel body is instantiated once
        const int col = static_cast<int>(w / a.ns);
        const int z0 = static_cast<int>(w - static_cast<int64_t>(col) * a.ns);
        const int z1 = static_cast<int>(min(static_cast<int64_t>(a.ns), z0 + (we - w)));
        ok = sweep_tile<D, R, T, VY, S, TX, TY, SH, CHK, P>(tmap, a, col, z0, z1, smem);
        w += z1 - z0;
    }
    return ok;
}

// ------------------------------------------------------------------ kernels
// One pass over the grid: block b sweeps its planes of the tile columns (sweep_block).
template <int D, int R, int T, int VY, typename S, int TX, int TY, bool SH, bool CHK, int P>
__global__ void __launch_bounds__(TX *TY)
    sweep_kernel(const __grid_constant__ CUtensorMap tmap, const __grid_constant__ SweepArgs a)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    sweep_block<D, R, T, VY, S, TX, TY, SH, CHK, P>(&tmap, a, static_cast<int>(blockIdx.x), smem);
}

// Persistent sweep of many grids of one kernel class, all passes, from a device tile
// queue.  Queue order is pass-major over the grids, so every tile a block waits for was
// taken earlier by a running block: pass p of grid g starts a tile only after all tiles
// of its pass p-1 are counted done (bounded spin; on expiry the status word is set and
// the block stops).
struct BatchTask {
    int prev;             // task whose output this task reads (-1 for a grid's first pass)
    int ntiles;           // tiles of this task
    int first;            // queue index of its first tile
};

struct BatchArgs {
    const SweepArgs *args;      // per task
    const CUtensorMap *maps;    // per task (3D)
    const BatchTask *tasks;
    int *done;                  // per task: tiles finished
    int *head;                  // next queue index
    unsigned *status;
    int ntasks, total;          // tasks, queue length
    int timeout_ms;
    int fault_task;             // test hook: this task never reports its tiles done (< 0: off)
};

__device__ __forceinline__ int ld_acquire(const int *p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void fence_proxy_async_global()
{
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

template <int D, int R, int T, int VY, typename S, int TX, int TY, bool SH, bool CHK, int P>
__global__ void __launch_bounds__(TX *TY)
    sweep_persistent(const __grid_constant__ BatchArgs B)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ int s_q, s_ok;
    const int tid = threadIdx.y * TX + threadIdx.x;
    for (;;) {
        if (tid == 0) s_q = atomicAdd(B.head, 1);
        __syncthreads();
        const int q = s_q;
        if (q >= B.total) break;
        // task of queue index q (binary search on first-tile indices)
        int lo = 0, hi = B.ntasks - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) / 2;
            if (B.tasks[mid].first <= q) lo = mid;
            else hi = mid - 1;
        }
        const int task = lo;
        const BatchTask tk = B.tasks[task];
        if (tid == 0) {
            int ok = 1;
            if (tk.prev >= 0) {
                const int need = B.tasks[tk.prev].ntiles;
                const int *cnt = B.done + tk.prev;
                if (ld_acquire(cnt) < need) {
                    const uint64_t t0 = global_ns();
                    const uint64_t lim = static_cast<uint64_t>(B.timeout_ms) * 1000000ull;
                    while (ld_acquire(cnt) < need) {
                        if (global_ns() - t0 > lim) {
                            ok = 0;
                            atomicOr(B.status, kStatusTimeout);
                            break;
                        }
                        __nanosleep(256);
                    }
                }
                // the input was written by other blocks' generic stores; the tile reads it with TMA
                fence_proxy_async_global();
            }
            s_ok = ok;
        }
        __syncthreads();
        if (!s_ok) break;
        const SweepArgs a = B.args[task];
        const bool done = sweep_block<D, R, T, VY, S, TX, TY, SH, CHK, P>(D == 3 ? B.maps + task : nullptr, a, q - tk.first, smem);
        __syncthreads();
        if (tid == 0 && task != B.fault_task) {
            __threadfence();
            fence_proxy_async_global();
            atomicAdd(B.done + task, 1);
        }
        if (!done) break;
    }
}

}  // namespace stn
