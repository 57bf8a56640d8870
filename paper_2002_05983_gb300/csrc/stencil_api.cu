// C ABI of the sweep library: argument checks, schedule planning, the
// multi-pass driver (ceil(iters / t) passes ping-ponging between the
// caller's output and a handle-owned scratch grid) and kernel launches.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <mutex>
#include <new>
#include <sstream>
#include <string>
#include <vector>

#include <cudaTypedefs.h>

#include "naive.h"
#include "registry.h"
#include "stencil.h"
#include "sweep_kernel.cuh"

struct stencil_plan {
    int dim = 0, r = 0, K = 0;
    int shared = 0;              // 1: one coefficient per distance (K = r + 1)
    int checked = 0;             // 1: bounds-checked kernel instantiations (stencil_set_checked)
    int kind() const { return shared + 2 * checked; }   // registry key of the kernel variant
    float c[stn::kMaxK] = {};
    void *scratch = nullptr;     // second grid of the ping-pong between passes
    size_t scratch_bytes = 0;
    int scratch_dev = -1;
    void *dev_in = nullptr;      // device copies for stencil_run_host
    void *dev_out = nullptr;
    size_t host_bytes = 0;
    int host_dev = -1;
    int fault_plane = -1;
    int timeout_ms = 2000;
    struct Tuned {
        int64_t nx, ny, nz;
        int dtype;
        stencil_schedule s;
    };
    std::vector<Tuned> tuned;   // schedules stored by stencil_tune
    struct ModelPick {
        int64_t nx, ny, nz;
        int dtype;
        unsigned gen;           // cost-model generation the pick was made with
        stencil_schedule s;
    };
    mutable std::vector<ModelPick> model_picks;   // default picks proposed by the active cost model
};

namespace {

thread_local int g_last_cuda_error = 0;

// With STENCIL_DEBUG set in the environment, failing CUDA calls are reported on stderr.
int cuda_fail(cudaError_t e, int line = 0)
{
    g_last_cuda_error = static_cast<int>(e);
    (void)cudaGetLastError();
    if (line && std::getenv("STENCIL_DEBUG"))
        std::fprintf(stderr, "stencil: CUDA error %d (%s) at stencil_api.cu:%d\n", static_cast<int>(e),
                     cudaGetErrorString(e), line);
    return e == cudaErrorMemoryAllocation ? STENCIL_ERR_OOM : STENCIL_ERR_CUDA;
}

#define CK(call)                                             \
    do {                                                     \
        cudaError_t e_ = (call);                             \
        if (e_ != cudaSuccess) return cuda_fail(e_, __LINE__); \
    } while (0)

int elem_bytes(int dtype) { return dtype == STENCIL_F32 ? 4 : 2; }

// ---------------------------------------------------------------- kernels
struct Registry {
    std::vector<stn::KernelEntry> all;
    Registry()
    {
        using L = int (*)(const stn::KernelEntry **);
        const L lists[] = {stn::list_2d_f32_r1,  stn::list_2d_f32_r2,  stn::list_2d_f32_r3,
                           stn::list_2d_f32_r4,  stn::list_3d_f32_r1,  stn::list_3d_f32_r2,
                           stn::list_3d_f32_r3,  stn::list_3d_f32_r4,  stn::list_2d_bf16_r1,
                           stn::list_2d_bf16_r2, stn::list_2d_bf16_r3, stn::list_2d_bf16_r4,
                           stn::list_3d_bf16_r1, stn::list_3d_bf16_r2, stn::list_3d_bf16_r3,
                           stn::list_3d_bf16_r4, stn::list_2d_f16_r1,  stn::list_2d_f16_r2,
                           stn::list_2d_f16_r3,  stn::list_2d_f16_r4,  stn::list_3d_f16_r1,
                           stn::list_3d_f16_r2,  stn::list_3d_f16_r3,  stn::list_3d_f16_r4,
                           stn::list_2d_f32_r5,  stn::list_2d_f32_r6,  stn::list_3d_f32_r5,
                           stn::list_3d_f32_r6,  stn::list_2d_bf16_r5, stn::list_2d_bf16_r6,
                           stn::list_3d_bf16_r5, stn::list_3d_bf16_r6, stn::list_2d_f16_r5,
                           stn::list_2d_f16_r6,  stn::list_3d_f16_r5,  stn::list_3d_f16_r6,
                           stn::list_2d_f32sh,   stn::list_3d_f32sh,   stn::list_checked,  stn::list_2d_f32_p2,
                           stn::list_2d_bf16_p2, stn::list_2d_f16_p2,  stn::list_2d_p4};
        for (L f : lists) {
            const stn::KernelEntry *e = nullptr;
            const int n = f(&e);
            all.insert(all.end(), e, e + n);
        }
    }
    // tx / ty = 0: the default block shape (the first listed for that degree); p: planes per step
    const stn::KernelEntry *find(int dim, int r, int t, int vy, int dtype, int sh, int tx = 0, int ty = 0,
                                 int p = 1) const
    {
        for (const auto &e : all)
            if (e.dim == dim && e.r == r && e.t == t && (dim == 2 || e.vy == vy) && e.dtype == dtype &&
                e.sh == sh && (!tx || e.tx == tx) && (dim == 2 || !ty || e.ty == ty) && e.p == p)
                return &e;
        return nullptr;
    }
    int max_t(int dim, int r, int dtype, int vy, int sh, int p = 1) const
    {
        int m = 0;
        for (const auto &e : all)
            if (e.dim == dim && e.r == r && e.dtype == dtype && (dim == 2 || e.vy == vy) && e.sh == sh && e.p == p)
                m = std::max(m, e.t);
        return m;
    }
};

const Registry &registry()
{
    static Registry reg;
    return reg;
}

// Functions whose shared-memory limit has been raised to the device maximum.
std::mutex g_attr_mu;
std::vector<const void *> g_attr_done;

std::vector<int> g_attr_regs;   // registers per thread of each prepared function

int prepare_fn(const void *fn, int max_smem, int *regs = nullptr)
{
    std::lock_guard<std::mutex> lk(g_attr_mu);
    const auto it = std::find(g_attr_done.begin(), g_attr_done.end(), fn);
    if (it != g_attr_done.end()) {
        if (regs) *regs = g_attr_regs[static_cast<size_t>(it - g_attr_done.begin())];
        return 0;
    }
    cudaFuncAttributes fa;
    CK(cudaFuncGetAttributes(&fa, fn));   // static shared memory counts against the same limit
    CK(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                            max_smem - static_cast<int>(fa.sharedSizeBytes)));
    g_attr_done.push_back(fn);
    g_attr_regs.push_back(fa.numRegs);
    if (regs) *regs = fa.numRegs;
    return 0;
}

struct DevInfo {
    int sms = 0, max_smem = 0;
    unsigned *status = nullptr;
};
std::mutex g_dev_mu;
DevInfo g_dev[64];

int device_info(DevInfo **out)
{
    int dev = 0;
    CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return STENCIL_ERR_NO_DEVICE;
    std::lock_guard<std::mutex> lk(g_dev_mu);
    DevInfo &d = g_dev[dev];
    if (!d.sms) {
        CK(cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev));
        CK(cudaDeviceGetAttribute(&d.max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
        void *p = nullptr;
        CK(cudaMalloc(&p, 256));
        CK(cudaMemset(p, 0, 256));
        CK(cudaDeviceSynchronize());
        d.status = static_cast<unsigned *>(p);
    }
    *out = &d;
    return 0;
}

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

// ------------------------------------------------------------- planning
int round_up(int a, int m) { return (a + m - 1) / m * m; }

struct Pass {
    const void *fn = nullptr;
    const stn::KernelEntry *e = nullptr;   // the kernel's registry entry
    int t = 0;
    int occ = 0;   // resident blocks per SM
    int regs = 0;  // registers per thread of the kernel
    int padin = 0; // input-plane x padding per side: 3D tensor-map box width 4*block.x + 2*padin
    dim3 grid, block;
    size_t smem = 0;
    stn::SweepArgs a{};
};

bool stream_applicable(int dtype, int64_t nx)
{
    return nx % (dtype == STENCIL_F32 ? 4 : 8) == 0;
}

void default_schedule(const stencil_plan *h, int64_t nx, int64_t ny, int64_t nz, int dtype,
                      stencil_schedule *s)
{
    (void)ny;
    (void)nz;
    const Registry &reg = registry();
    stencil_schedule d{};
    // shared-coefficient stencils have FP32 streaming kernels only; other storage runs naive
    const bool have = reg.max_t(h->dim, h->r, dtype, h->dim == 3 ? 2 : 1, h->kind()) > 0;
    d.kernel = (have && stream_applicable(dtype, nx)) ? STENCIL_KERNEL_STREAM : STENCIL_KERNEL_NAIVE;
    if (h->dim == 2) {
        // measured on 16384^2: radius 1 peaks at t = 4 with one row per step; radii 2-4 gain
        // 12-19 % from two rows per step (FP32 t = 3, 2, 2; 16-bit storage radius 3 at t = 3)
        static const int t2[stn::kMaxR + 1] = {0, 4, 3, 2, 2, 2, 2};
        static const int t2h[stn::kMaxR + 1] = {0, 4, 3, 3, 2, 2, 2};
        d.t = std::max(1, std::min(dtype == STENCIL_F32 ? t2[h->r] : t2h[h->r], reg.max_t(2, h->r, dtype, 1, h->kind())));
        d.threads_x = 128;
        d.threads_y = 1;
        d.rows_per_thread = 1;
        d.planes_per_step = h->r >= 2 && reg.find(2, h->r, d.t, 1, dtype, h->kind(), 128, 0, 2) ? 2 : 1;
    } else {
        d.t = h->r == 1 ? 2 : 1;
        // FP32 radius 3 and 4 (one level, packed two-lane arithmetic): 4 rows per thread
        // measured 670 / 613 against 654 / 591 GCell/s with 2 rows on 512^3
        const bool four = dtype == STENCIL_F32 && h->kind() == 0 && d.t == 1 && (h->r == 3 || h->r == 4) &&
                          reg.find(3, h->r, 1, 4, dtype, 0, 16, 8, 1) != nullptr;
        d.rows_per_thread = four ? 4 : 2;
        d.threads_x = 16;
        d.threads_y = 8;
        d.planes_per_step = 1;
    }
    d.seg = 0;
    d.prefetch = 0;
    *s = d;
}

// ---- persistent tuning cache: the file named by STENCIL_TUNE_CACHE holds one line per
// stored pick, "v2 <gpu> <dim> <r> <shared> <dtype> <nx> <ny> <nz> <kernel> <t> <threads_x>
// <threads_y> <rows> <seg> <prefetch> <planes_per_step>", the last line for a key winning
// (v1 lines, without the last field, are read as one plane per step).  A pick is keyed by
// the GPU's name and the problem (not the coefficients, which do not change the speed).
struct FileCacheEntry {
    std::string gpu;
    int dim, r, sh, dtype;
    int64_t nx, ny, nz;
    stencil_schedule s;
};
std::mutex g_fc_mu;
std::string g_fc_path;
std::vector<FileCacheEntry> g_fc;

bool gpu_name(std::string *out)
{
    static std::mutex mu;
    static std::string names[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return false;
    }
    std::lock_guard<std::mutex> lk(mu);
    if (names[dev].empty()) {
        cudaDeviceProp p;
        if (cudaGetDeviceProperties(&p, dev) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        std::string n = p.name;
        for (char &c : n)
            if (c == ' ' || c == '\t') c = '_';
        names[dev] = n;
    }
    *out = names[dev];
    return true;
}

// (Re)load the cache when STENCIL_TUNE_CACHE names another file; caller holds g_fc_mu.
const char *fc_sync()
{
    const char *path = std::getenv("STENCIL_TUNE_CACHE");
    if (!path || !*path) return nullptr;
    if (g_fc_path != path) {
        g_fc.clear();
        g_fc_path = path;
        std::ifstream f(path);
        std::string line;
        while (std::getline(f, line)) {
            std::istringstream is(line);
            std::string v;
            FileCacheEntry e{};
            if (!(is >> v >> e.gpu >> e.dim >> e.r >> e.sh >> e.dtype >> e.nx >> e.ny >> e.nz >> e.s.kernel >> e.s.t >>
                  e.s.threads_x >> e.s.threads_y >> e.s.rows_per_thread >> e.s.seg >> e.s.prefetch) ||
                (v != "v1" && v != "v2"))
                continue;   // not a cache line
            e.s.planes_per_step = 1;
            if (v == "v2" && !(is >> e.s.planes_per_step)) continue;
            g_fc.push_back(e);
        }
    }
    return path;
}

bool fc_lookup(const stencil_plan *h, int64_t nx, int64_t ny, int64_t nz, int dtype, stencil_schedule *out)
{
    std::string gpu;
    if (!std::getenv("STENCIL_TUNE_CACHE") || !gpu_name(&gpu)) return false;
    std::lock_guard<std::mutex> lk(g_fc_mu);
    if (!fc_sync()) return false;
    bool hit = false;
    for (const auto &e : g_fc)
        if (e.gpu == gpu && e.dim == h->dim && e.r == h->r && e.sh == h->kind() && e.dtype == dtype && e.nx == nx &&
            e.ny == ny && e.nz == nz) {
            *out = e.s;
            hit = true;
        }
    return hit;
}

void fc_store(const stencil_plan *h, int64_t nx, int64_t ny, int64_t nz, int dtype, const stencil_schedule &s)
{
    std::string gpu;
    if (!std::getenv("STENCIL_TUNE_CACHE") || !gpu_name(&gpu)) return;
    std::lock_guard<std::mutex> lk(g_fc_mu);
    const char *path = fc_sync();
    if (!path) return;
    std::ofstream f(path, std::ios::app);
    f << "v2 " << gpu << ' ' << h->dim << ' ' << h->r << ' ' << h->kind() << ' ' << dtype << ' ' << nx << ' ' << ny
      << ' ' << nz << ' ' << s.kernel << ' ' << s.t << ' ' << s.threads_x << ' ' << s.threads_y << ' '
      << s.rows_per_thread << ' ' << s.seg << ' ' << s.prefetch << ' ' << s.planes_per_step << '\n';
    g_fc.push_back({gpu, h->dim, h->r, h->kind(), dtype, nx, ny, nz, s});
}

// The cost model that proposes default schedules (stencil_use_cost_model), and a generation
// count that retires the picks made with an earlier model.
std::mutex g_model_mu;
stencil_model_handle g_model = nullptr;
unsigned g_model_gen = 0;

// The schedule stencil_run uses when the caller gives none: a pick stored on the handle,
// else one in the tuning-cache file, else the active cost model's proposal, else the
// library's rule.
void chosen_schedule(const stencil_plan *h, int64_t nx, int64_t ny, int64_t nz, int dtype, stencil_schedule *s)
{
    default_schedule(h, nx, ny, nz, dtype, s);
    bool picked = fc_lookup(h, nx, ny, nz, dtype, s);
    for (const auto &tu : h->tuned)
        if (tu.nx == nx && tu.ny == ny && tu.nz == nz && tu.dtype == dtype) {
            *s = tu.s;
            picked = true;
        }
    if (picked) return;
    stencil_model_handle m = nullptr;
    unsigned gen = 0;
    {
        std::lock_guard<std::mutex> lk(g_model_mu);
        m = g_model;
        gen = g_model_gen;
    }
    if (!m || s->kernel != STENCIL_KERNEL_STREAM) return;
    for (const auto &mp : h->model_picks)
        if (mp.gen == gen && mp.nx == nx && mp.ny == ny && mp.nz == nz && mp.dtype == dtype) {
            *s = mp.s;
            return;
        }
    stencil_schedule pick;
    if (stencil_tune(const_cast<stencil_plan *>(h), nx, ny, nz, dtype, STENCIL_TUNE_MODEL, m, 0, &pick, nullptr, 0,
                     nullptr) != STENCIL_OK)
        return;   // keep the library's rule
    *s = pick;
    h->model_picks.push_back({nx, ny, nz, dtype, gen, pick});
}

// Fill one pass of temporal degree t.  Pointers are set by the caller.
int plan_pass(const stencil_plan *h, int64_t nx, int64_t ny, int64_t nz, int dtype, int t,
              const stencil_schedule &s, const DevInfo &dev, Pass &ps, bool batched = false)
{
    const int D = h->dim, R = h->r;
    const int vy = D == 3 ? s.rows_per_thread : 1;
    int pps = D == 2 && s.planes_per_step ? s.planes_per_step : 1;
    const stn::KernelEntry *e = registry().find(D, R, t, vy, dtype, h->kind(), s.threads_x, D == 3 ? s.threads_y : 0, pps);
    while (!e && pps > 1) {   // a degree compiled with fewer rows per step (e.g. a remainder pass)
        pps /= 2;
        e = registry().find(D, R, t, vy, dtype, h->kind(), s.threads_x, 0, pps);
    }
    if (!e) return STENCIL_ERR_UNSUPPORTED;
    // the prefetch depth is a property of the degree-t kernel; a pass of another degree (the
    // remainder, or fewer iterations than t) runs its own kernel's
    if (s.prefetch && t == s.t && s.prefetch != e->pf) return STENCIL_ERR_UNSUPPORTED;
    if (e->smem > static_cast<size_t>(dev.max_smem)) return STENCIL_ERR_UNSUPPORTED;
    int regs = 0;
    int rc = prepare_fn(e->fn, dev.max_smem, &regs);
    if (rc) return rc;
    int occ = 0;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, e->fn, e->tx * e->ty, e->smem));
    if (occ < 1) return STENCIL_ERR_UNSUPPORTED;

    const int64_t ntx = (nx + e->cx - 1) / e->cx;
    const int64_t nty = D == 3 ? (ny + e->cy - 1) / e->cy : 1;
    const int64_t ns = D == 3 ? nz : ny;
    const int64_t tiles = ntx * nty;
    const int64_t slots = static_cast<int64_t>(dev.sms) * occ;
    const int64_t minseg = std::max<int64_t>(64, 8 * t * (2 * R + pps));
    // Two block orders.  Slabs: the stream axis is cut into slabs of seg planes,
    // the tiles of one slab in consecutive blocks, so blocks that run together
    // read neighbouring tiles of the same rows/planes (DRAM locality, shared halo
    // reads in L2).  Strips end to end (2D kernels that are issue-bound: a long
    // loop body, or t >= 5): the strips' rows laid end to end are split into equal
    // ranges, one per resident block slot for long bodies, so no SM waits on a
    // partly filled last wave.  (Measured on 16384^2: slabs win at t <= 4 with
    // short bodies by 4-10 %, strips win by 3-25 % otherwise.)
    const int64_t body = static_cast<int64_t>(2 * R + 1) * t * 4 * (4 * R + 1);
    const bool flat = D == 2 && (body > 400 || t >= 5);
    const int64_t W = tiles * ns;
    int64_t seg = s.seg;
    if (seg <= 0) {
        if (!flat) {
            // >= 4 waves (dynamic balance of edge tiles), segments long against the fill
            const int64_t want = (4 * slots + tiles - 1) / tiles;
            seg = std::max<int64_t>((ns + want - 1) / want, minseg);
        } else if (batched) {
            // other grids fill the device: segments long against the pipeline fill
            seg = std::max<int64_t>((W + 4 * slots - 1) / (4 * slots), minseg);
        } else {
            seg = (W + slots - 1) / slots;
            // short bodies: several equal waves of ~200-row blocks keep blocks out of phase
            if (body <= 400) seg = std::min<int64_t>(seg, std::max<int64_t>(192, (W + 8 * slots - 1) / (8 * slots)));
        }
    }
    seg = std::max<int64_t>(seg, 1);
    seg = std::min<int64_t>(seg, flat ? W : ns);
    const int64_t nblk = flat ? (W + seg - 1) / seg : tiles * ((ns + seg - 1) / seg);
    if (nblk > 0x7fffffffLL || seg > 0x7fffffffLL) return STENCIL_ERR_UNSUPPORTED;

    ps.fn = e->fn;
    ps.e = e;
    ps.t = t;
    ps.occ = occ;
    ps.regs = regs;
    ps.grid = dim3(static_cast<unsigned>(nblk));
    ps.block = dim3(e->tx, e->ty);
    ps.smem = e->smem;
    ps.padin = e->padin;
    stn::SweepArgs &a = ps.a;
    a.nx = static_cast<int>(nx);
    a.ny = static_cast<int>(ny);
    a.nz = static_cast<int>(nz);
    a.ns = static_cast<int>(ns);
    a.seg = static_cast<int>(seg);
    a.flat = flat ? 1 : 0;
    a.ntx = static_cast<int>(ntx);
    a.nty = static_cast<int>(nty);
    a.timeout_ms = h->timeout_ms;
    a.fault_plane = h->fault_plane;
    a.status = dev.status;
    std::memcpy(a.c, h->c, sizeof(float) * h->K);
    for (int k = 0; k < h->K; ++k) a.cc[2 * k] = a.cc[2 * k + 1] = h->c[k];
    return 0;
}

int encode_map(CUtensorMap *m, const void *ptr, int64_t nx, int64_t ny, int64_t nz, int dtype,
               int box_w, int box_h)
{
    auto enc = tensor_map_encoder();
    if (!enc) return STENCIL_ERR_CUDA;
    const int es = elem_bytes(dtype);
    cuuint64_t dims[3] = {static_cast<cuuint64_t>(nx), static_cast<cuuint64_t>(ny),
                          static_cast<cuuint64_t>(nz)};
    cuuint64_t strides[2] = {static_cast<cuuint64_t>(nx * es), static_cast<cuuint64_t>(nx * ny * es)};
    cuuint32_t box[3] = {static_cast<cuuint32_t>(box_w), static_cast<cuuint32_t>(box_h), 1};
    cuuint32_t estr[3] = {1, 1, 1};
    const CUtensorMapDataType dt = dtype == STENCIL_F32    ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                   : dtype == STENCIL_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                           : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
    const CUresult r = enc(m, dt, 3, const_cast<void *>(ptr), dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        g_last_cuda_error = static_cast<int>(r);
        if (std::getenv("STENCIL_DEBUG"))
            std::fprintf(stderr, "stencil: cuTensorMapEncodeTiled error %d (box %d x %d, dims %lld %lld %lld)\n",
                         static_cast<int>(r), box_w, box_h, static_cast<long long>(nx), static_cast<long long>(ny),
                         static_cast<long long>(nz));
        return STENCIL_ERR_CUDA;
    }
    return 0;
}

int ensure_scratch(stencil_plan *h, size_t bytes)
{
    int dev = 0;
    CK(cudaGetDevice(&dev));
    if (h->scratch && (h->scratch_bytes < bytes || h->scratch_dev != dev)) {
        CK(cudaDeviceSynchronize());
        CK(cudaFree(h->scratch));
        h->scratch = nullptr;
        h->scratch_bytes = 0;
    }
    if (!h->scratch) {
        CK(cudaMalloc(&h->scratch, bytes));
        h->scratch_bytes = bytes;
        h->scratch_dev = dev;
    }
    return 0;
}

bool ranges_overlap(const void *a, size_t na, const void *b, size_t nb)
{
    const uintptr_t x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
    return x < y + nb && y < x + na;
}

bool overlap(const void *a, const void *b, size_t n)
{
    const uintptr_t x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
    return x < y + n && y < x + n;
}

int check_problem(const stencil_plan *h, const void *in, const void *out, int64_t nx, int64_t ny,
                  int64_t nz, int iters, int dtype)
{
    if (!h || !in || !out) return STENCIL_ERR_INVALID_ARG;
    if (nx <= 0 || ny <= 0 || nz <= 0 || iters < 0) return STENCIL_ERR_INVALID_ARG;
    if (h->dim == 2 && nz != 1) return STENCIL_ERR_INVALID_ARG;
    if (dtype < STENCIL_F32 || dtype > STENCIL_F16) return STENCIL_ERR_INVALID_ARG;
    if (nx > 0x7fffffff || ny > 0x7fffffff || nz > 0x7fffffff) return STENCIL_ERR_INVALID_ARG;
    const size_t bytes = static_cast<size_t>(nx * ny * nz) * elem_bytes(dtype);
    if (overlap(in, out, bytes)) return STENCIL_ERR_ALIAS;
    return 0;
}

int launch_naive(const stencil_plan *h, const void *src, void *dst, int64_t nx, int64_t ny,
                 int64_t nz, int dtype, cudaStream_t st, const DevInfo &dev)
{
    const void *fn = stn::naive_fn(h->dim, h->r, dtype, h->shared);
    if (!fn) return STENCIL_ERR_UNSUPPORTED;
    stn::NaiveArgs na{};
    na.nx = static_cast<int>(nx);
    na.ny = static_cast<int>(ny);
    na.nz = static_cast<int>(nz);
    std::memcpy(na.c, h->c, sizeof(float) * h->K);
    const int64_t n = nx * ny * nz;
    const int64_t want = (n + 255) / 256;
    const unsigned blocks = static_cast<unsigned>(std::min<int64_t>(want, static_cast<int64_t>(dev.sms) * 32));
    void *args[] = {const_cast<void **>(&src), &dst, &na};
    CK(cudaLaunchKernel(fn, dim3(blocks), dim3(256), args, 0, st));
    return 0;
}

int run_impl(stencil_plan *h, const void *in, void *out, int64_t nx, int64_t ny, int64_t nz,
             int iters, int dtype, cudaStream_t st, const stencil_schedule *user)
{
    int rc = check_problem(h, in, out, nx, ny, nz, iters, dtype);
    if (rc) return rc;
    DevInfo *dev = nullptr;
    rc = device_info(&dev);
    if (rc) return rc;
    const size_t bytes = static_cast<size_t>(nx * ny * nz) * elem_bytes(dtype);
    if (iters == 0) {
        CK(cudaMemcpyAsync(out, in, bytes, cudaMemcpyDeviceToDevice, st));
        return 0;
    }
    stencil_schedule s;
    chosen_schedule(h, nx, ny, nz, dtype, &s);
    if (user) {
        if (user->kernel < 0 || user->kernel > STENCIL_KERNEL_NAIVE) return STENCIL_ERR_INVALID_ARG;
        if (user->kernel) s.kernel = user->kernel;
        if (user->t) s.t = user->t;
        if (user->threads_x) s.threads_x = user->threads_x;
        if (user->threads_y) s.threads_y = user->threads_y;
        if (user->rows_per_thread) s.rows_per_thread = user->rows_per_thread;
        if (user->seg) s.seg = user->seg;
        if (user->prefetch) s.prefetch = user->prefetch;
        if (user->planes_per_step) s.planes_per_step = user->planes_per_step;
        if (s.t < 0 || s.seg < 0 || s.prefetch < 0 || s.planes_per_step < 0 || s.planes_per_step > 4)
            return STENCIL_ERR_INVALID_ARG;
        if (h->dim == 3 && user->t && !user->rows_per_thread)
            s.rows_per_thread = 2;
    }
    const bool aligned = (reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(out)) % 16 == 0;
    const bool streamable = stream_applicable(dtype, nx) && aligned;
    if (s.kernel == STENCIL_KERNEL_STREAM && !streamable) return STENCIL_ERR_UNSUPPORTED;
    if (s.kernel == STENCIL_KERNEL_AUTO) s.kernel = streamable ? STENCIL_KERNEL_STREAM : STENCIL_KERNEL_NAIVE;

    // passes: full passes of degree t, then the remainder
    std::vector<int> degrees;
    const int t = s.kernel == STENCIL_KERNEL_NAIVE ? 1 : std::max(1, std::min(s.t, iters));
    for (int done = 0; done < iters; done += t) degrees.push_back(std::min(t, iters - done));
    const int L = static_cast<int>(degrees.size());
    if (L > 1) {
        rc = ensure_scratch(h, bytes);
        if (rc) return rc;
    }
    std::vector<Pass> plans;
    if (s.kernel == STENCIL_KERNEL_STREAM) {
        for (int j = 0; j < L; ++j) {
            if (j > 0 && degrees[j] == degrees[j - 1]) {
                plans.push_back(plans.back());
                continue;
            }
            Pass ps;
            rc = plan_pass(h, nx, ny, nz, dtype, degrees[j], s, *dev, ps);
            if (rc) return rc;
            plans.push_back(ps);
        }
    }
    const void *src = in;
    for (int j = 0; j < L; ++j) {
        void *dst = ((L - 1 - j) % 2 == 0) ? out : h->scratch;
        if (s.kernel == STENCIL_KERNEL_NAIVE) {
            rc = launch_naive(h, src, dst, nx, ny, nz, dtype, st, *dev);
            if (rc) return rc;
        } else {
            Pass &ps = plans[j];
            ps.a.in = src;
            ps.a.out = dst;
            CUtensorMap map;
            std::memset(&map, 0, sizeof(map));
            if (h->dim == 3) {
                rc = encode_map(&map, src, nx, ny, nz, dtype, 4 * static_cast<int>(ps.block.x) + 2 * ps.padin,
                                static_cast<int>(ps.block.y) * s.rows_per_thread + 2 * h->r);
                if (rc) return rc;
            }
            void *args[] = {&map, &ps.a};
            CK(cudaLaunchKernel(ps.fn, ps.grid, ps.block, args, ps.smem, st));
        }
        src = dst;
    }
    return 0;
}

// ------------------------------------------------------------------------
// Schedule tuner: candidates, analytic model, features.
// Issue-slot model of the streaming kernel, calibrated with the profiled kernels' ncu opcode
// counts and their measured rates: per step and time level a thread issues its 4*VY*P cells'
// FP32 chains (one FMUL and 2*D*r FFMA per cell) plus bookkeeping (neighbour loads, ring stores,
// ring addressing, the copy wait and the barrier: 2D about 2.6 + 4.5 r + 13.9 P instructions,
// 10 P more for level 1's widening loads from a 16-bit ring; 3D the y/x neighbour loads of every
// row and, for shifting queues, the register moves); warps issue at kIssueEff of the SM's rate
// once 16 warps per SM hide the latencies.
constexpr double kLaneIssuePerSmPerClk = 128.0;   // 4 schedulers x 32 lanes
constexpr double kSmClockHz = 2.07e9;             // maximum SM clock (held under load, clock samples)
constexpr double kIssueEff = 0.64;                // issue share reached with >= 16 resident warps per SM
constexpr double kFullWarps = 16.0;               // resident warps per SM below which latency is exposed
constexpr double kHbmBytesPerS = 6787.6e9 * 0.92; // measured copy bandwidth, achievable share
// Resolve every field of a schedule for a problem (the pass of degree t).
int resolve(const stencil_plan *h, int64_t nx, int64_t ny, int64_t nz, int dtype, stencil_schedule s,
            const DevInfo &dev, stencil_schedule &out, Pass &ps)
{
    int rc = plan_pass(h, nx, ny, nz, dtype, s.t, s, dev, ps);
    if (rc) return rc;
    out = s;
    out.kernel = STENCIL_KERNEL_STREAM;
    out.threads_x = static_cast<int>(ps.block.x);
    out.threads_y = static_cast<int>(ps.block.y);
    out.seg = ps.a.seg;
    out.prefetch = ps.e->pf;
    out.planes_per_step = ps.e->p;
    if (h->dim == 2) out.rows_per_thread = 1;
    return 0;
}

// Analytic time per cell update (ns) of a resolved schedule: the larger of the HBM time
// (2 s bytes per cell per pass) and the issue time of the blocks, which run in waves of
// SMs x occupancy.
double analytic_ns(const stencil_plan *h, int64_t nx, int64_t ny, int64_t nz, int dtype, const stencil_schedule &s,
                   int occ, int sms)
{
    const int D = h->dim, R = h->r, t = s.t;
    const stn::KernelEntry *e = registry().find(D, R, t, D == 3 ? s.rows_per_thread : 1, dtype, h->kind(), s.threads_x,
                                                s.threads_y, D == 2 && s.planes_per_step ? s.planes_per_step : 1);
    if (!e) return 1e9;
    const double es = elem_bytes(dtype);
    const double N = static_cast<double>(nx) * ny * nz;
    const double tiles = std::ceil(nx / static_cast<double>(e->cx)) * (D == 3 ? std::ceil(ny / static_cast<double>(e->cy)) : 1.0);
    const double ns_axis = D == 3 ? static_cast<double>(nz) : static_cast<double>(ny);
    const double nblk = std::ceil(tiles * ns_axis / s.seg);
    const int P = e->p, VY = e->vy, NV = (R + 3) / 4;
    const double cells = 4.0 * VY * P;                               // per thread, level and step
    // FP32 instructions per cell: 2*D*r + 1 (both coefficient forms); the 3D FP32 one-level
    // kernels of radius 3 and 4 run two cells per packed instruction except the x terms of
    // odd distance: 1/2 for the centre, 3 per even and 4 per odd distance
    const bool packed = D == 3 && t == 1 && dtype == STENCIL_F32 && !h->shared && (R == 3 || R == 4);
    double fpc = 2.0 * D * R + 1.0;
    if (packed) {
        fpc = 0.5;
        for (int i = 1; i <= R; ++i) fpc += (i % 2 == 0) ? 3.0 : 4.0;
    }
    const double fp = cells * fpc;
    const double book = (D == 2 ? 2.6 + 4.5 * R + 13.9 * P
                                : 20.0 + 2.0 * (2.0 * R + 2.0 * NV) * VY + (e->rot ? 0.0 : 6.0 * VY * e->qp / e->u)) +
                        (es == 2 ? 10.0 * P / t : 0.0);   // level 1 of t widens its 16-bit neighbour loads
    // stream planes of a block: its segment, the r*t halo planes and the pipeline fill
    const double lagT = std::max(R, P) + (t - 1) * (P + std::max(R, P));
    const double steps = (std::min<double>(s.seg, ns_axis) + 2.0 * t * R + lagT) / P;
    const double instr = static_cast<double>(e->tx) * e->ty * steps * t * (fp + book);
    const double slots = static_cast<double>(sms) * std::max(occ, 1);
    const double waves = std::ceil(nblk / slots);
    const double warps = static_cast<double>(occ) * e->tx * e->ty / 32.0;
    const double eff = kIssueEff * std::min(1.0, warps / kFullWarps);
    const double t_issue = waves * instr * std::max(occ, 1) / (kLaneIssuePerSmPerClk * kSmClockHz * std::max(eff, 0.02));
    const double t_mem = N * 2.0 * es / kHbmBytesPerS;
    return std::max(t_issue, t_mem) / (N * t) * 1e9;
}

void features_of(const stencil_plan *h, int64_t nx, int64_t ny, int64_t nz, int dtype, const stencil_schedule &s,
                 const Pass &ps, double analytic, int sms, float *f)
{
    const int occ = ps.occ;
    const stn::KernelEntry *e = ps.e;
    f[0] = static_cast<float>(h->dim);
    f[1] = static_cast<float>(h->r);
    f[2] = static_cast<float>(std::log2(static_cast<double>(nx)));
    f[3] = static_cast<float>(std::log2(static_cast<double>(ny)));
    f[4] = static_cast<float>(std::log2(static_cast<double>(nz)));
    f[5] = static_cast<float>(elem_bytes(dtype));
    f[6] = static_cast<float>(s.t);
    const int vy = h->dim == 3 ? s.rows_per_thread : 1;
    f[7] = static_cast<float>(occ * s.threads_x * s.threads_y / 32);   // resident warps per SM
    f[8] = static_cast<float>(h->dim == 3 ? s.threads_y * vy : 1);
    // size of the unrolled loop body: queue period x levels x cells x FMA per cell
    f[9] = static_cast<float>(std::log2(static_cast<double>(e->qp) * s.t * 4 * vy * (2 * h->dim * h->r + 1)));
    f[10] = static_cast<float>(std::log2(static_cast<double>(s.seg)));
    f[11] = static_cast<float>(std::log2(analytic));
    // work partition: block order (strips end to end or slabs) and waves of resident blocks
    f[12] = static_cast<float>(ps.a.flat);
    f[13] = static_cast<float>(std::log2(static_cast<double>(ps.grid.x) / (static_cast<double>(sms) * std::max(occ, 1))));
    // rows per step, halo redundancy (thread region over compute tile), registers, shared memory
    f[14] = static_cast<float>(e->p);
    const double reg = 4.0 * e->tx * (h->dim == 3 ? e->ty * e->vy : 1);
    f[15] = static_cast<float>(std::log2(reg / (static_cast<double>(e->cx) * e->cy)));
    f[16] = static_cast<float>(ps.regs) / 64.0f;
    f[17] = static_cast<float>(std::log2(static_cast<double>(e->smem) / 1024.0));
}

// Candidate schedules (unresolved) of a problem.
int candidates(const stencil_plan *h, int64_t ny, int64_t nz, int dtype, stencil_schedule *out, int cap)
{
    int n = 0;
    const int64_t ns = h->dim == 3 ? nz : ny;
    const int segs2[] = {0, 128, 256, 512, 1024};
    const int segs3[] = {0, 32, 64, 128, 256};
    const int *segs = h->dim == 2 ? segs2 : segs3;
    for (int vy : {2, 4}) {
        if (h->dim == 2 && vy == 4) break;
        const int tmax = registry().max_t(h->dim, h->r, dtype, h->dim == 3 ? vy : 1, h->kind());
        for (int t = 1; t <= tmax; ++t)
            for (int pps = 1; pps <= (h->dim == 2 ? 2 : 1); ++pps) {
                if (pps == 2 && !registry().find(2, h->r, t, 1, dtype, h->kind(), 0, 0, 2)) continue;
                for (int k = 0; k < 5; ++k) {
                    if (segs[k] > ns) continue;
                    if (n >= cap) return n;
                    stencil_schedule s{};
                    s.kernel = STENCIL_KERNEL_STREAM;
                    s.t = t;
                    s.rows_per_thread = h->dim == 3 ? vy : 1;
                    s.seg = segs[k];
                    s.planes_per_step = pps;
                    out[n++] = s;
                }
            }
    }
    return n;
}

// ------------------------------------------------------------------------
// Batched persistent sweeps: plans, device task tables and cached CUDA graphs.
struct BatchClass {
    const void *pfn = nullptr;
    int phase = 0;                 // 0: full passes of every grid; 1: remainder passes
    dim3 grid, block;
    size_t smem = 0;
    stn::BatchArgs args{};
    void *dev_args = nullptr, *dev_maps = nullptr, *dev_tasks = nullptr, *dev_done = nullptr;
};

struct BatchEntry {
    std::vector<char> key;
    std::vector<void *> scratch;   // one per item (null when a grid needs a single pass)
    std::vector<BatchClass> classes;
    cudaGraphExec_t exec = nullptr;
    int dev = -1;
};

std::mutex g_batch_mu;
std::vector<BatchEntry *> g_batch;   // most recent last

void free_entry(BatchEntry *e)
{
    cudaDeviceSynchronize();   // a replay may still use the tables
    if (e->exec) cudaGraphExecDestroy(e->exec);
    for (void *p : e->scratch)
        if (p) cudaFree(p);
    for (auto &c : e->classes) {
        for (void *p : {c.dev_args, c.dev_maps, c.dev_tasks, c.dev_done})
            if (p) cudaFree(p);
    }
    delete e;
}

std::vector<char> batch_key(const stencil_batch_item *items, int n, int dev)
{
    std::vector<char> k(sizeof(int) + sizeof(stencil_batch_item) * n);
    std::memcpy(k.data(), &dev, sizeof(int));
    std::memcpy(k.data() + sizeof(int), items, sizeof(stencil_batch_item) * n);
    for (int i = 0; i < n; ++i) {   // the handles' coefficients, schedules and test settings
        const stencil_plan *h = items[i].h;
        const char *c = reinterpret_cast<const char *>(h->c);
        k.insert(k.end(), c, c + sizeof(float) * h->K);
        int extra[3] = {h->fault_plane, h->timeout_ms, h->kind()};   // kind: shared / checked kernels
        k.insert(k.end(), reinterpret_cast<char *>(extra), reinterpret_cast<char *>(extra) + sizeof(extra));
        stencil_schedule sc;   // the schedule the batch will use for this grid
        chosen_schedule(h, items[i].nx, items[i].ny, items[i].nz, items[i].dtype, &sc);
        const char *b = reinterpret_cast<const char *>(&sc);
        k.insert(k.end(), b, b + sizeof(sc));
    }
    return k;
}

int build_batch(const stencil_batch_item *items, int n, const DevInfo &dev, cudaStream_t st, BatchEntry *E)
{
    // Every grid runs ceil(iters / t) passes at its own chosen degree t, like stencil_run:
    // L = iters / t full passes (phase 0), then one remainder pass of degree iters mod t
    // (phase 1).  Each pass becomes a task of the kernel class that sweeps it.
    struct Pass1 {
        int item, pass, phase;
        Pass ps;
    };
    std::vector<Pass1> passes;
    std::vector<int> npass(n, 0);
    for (int i = 0; i < n; ++i) {
        const stencil_batch_item &b = items[i];
        stencil_plan *h = b.h;
        stencil_schedule s;
        chosen_schedule(h, b.nx, b.ny, b.nz, b.dtype, &s);
        if (s.kernel != STENCIL_KERNEL_STREAM) return STENCIL_ERR_UNSUPPORTED;
        const int t = std::max(1, std::min(s.t, b.iters));
        const int full = b.iters / t, rem = b.iters % t;
        npass[i] = full + (rem ? 1 : 0);
        for (int p = 0; p < npass[i]; ++p) {
            Pass1 x;
            x.item = i;
            x.pass = p;
            x.phase = p < full ? 0 : 1;
            if (p == 0 || p == full) {
                const int rc = plan_pass(h, b.nx, b.ny, b.nz, b.dtype, p < full ? t : rem, s, dev, x.ps, true);
                if (rc) return rc;
                x.ps.a.timeout_ms = h->timeout_ms;
            } else {
                x.ps = passes.back().ps;
            }
            passes.push_back(x);
        }
    }
    // scratch grids (the second buffer of each grid's ping-pong)
    E->scratch.assign(n, nullptr);
    for (int i = 0; i < n; ++i)
        if (npass[i] > 1) {
            const stencil_batch_item &b = items[i];
            const size_t bytes = static_cast<size_t>(b.nx * b.ny * b.nz) * elem_bytes(b.dtype);
            CK(cudaMalloc(&E->scratch[i], bytes));
        }
    // kernel classes per phase; inside a class, tasks pass-major, largest grids first, so every
    // tile a block waits for was taken earlier by a running block of the same class
    for (int phase = 0; phase < 2; ++phase) {
        std::vector<const stn::KernelEntry *> kinds;
        for (const Pass1 &x : passes)
            if (x.phase == phase && std::find(kinds.begin(), kinds.end(), x.ps.e) == kinds.end())
                kinds.push_back(x.ps.e);
        for (const stn::KernelEntry *kind : kinds) {
            std::vector<const Pass1 *> mine;
            for (const Pass1 &x : passes)
                if (x.phase == phase && x.ps.e == kind) mine.push_back(&x);
            std::stable_sort(mine.begin(), mine.end(), [](const Pass1 *a, const Pass1 *b) {
                if (a->pass != b->pass) return a->pass < b->pass;
                return a->ps.grid.x > b->ps.grid.x;
            });
            std::vector<stn::SweepArgs> args;
            std::vector<CUtensorMap> maps;
            std::vector<stn::BatchTask> tasks;
            std::vector<int> last_task(n, -1);
            int total = 0, fault_task = -1, timeout = 2000;
            for (const Pass1 *x : mine) {
                const stencil_batch_item &b = items[x->item];
                const int L = npass[x->item], p = x->pass;
                void *scr = E->scratch[x->item];
                const void *src = p == 0 ? b.in : ((L - p) % 2 == 0 ? b.out : scr);
                void *dst = ((L - 1 - p) % 2 == 0) ? b.out : scr;
                stn::SweepArgs a = x->ps.a;
                a.in = src;
                a.out = dst;
                args.push_back(a);
                CUtensorMap m;
                std::memset(&m, 0, sizeof(m));
                if (b.h->dim == 3) {
                    const int rc = encode_map(&m, src, b.nx, b.ny, b.nz, b.dtype, 4 * kind->tx + 2 * kind->padin,
                                              kind->ty * kind->vy + 2 * b.h->r);
                    if (rc) return rc;
                }
                maps.push_back(m);
                stn::BatchTask tk;
                tk.prev = last_task[x->item];   // the grid's previous pass in this class (phase 0)
                tk.ntiles = static_cast<int>(x->ps.grid.x);
                tk.first = total;
                total += tk.ntiles;
                if (b.h->fault_plane == p && fault_task < 0) fault_task = static_cast<int>(tasks.size());
                timeout = b.h->timeout_ms;
                last_task[x->item] = static_cast<int>(tasks.size());
                tasks.push_back(tk);
            }
            E->classes.emplace_back();   // owned by E from here on: freed with it on any error below
            BatchClass &c = E->classes.back();
            c.pfn = kind->pfn;
            c.phase = phase;
            c.block = dim3(kind->tx, kind->ty);
            c.smem = kind->smem;
            int rc = prepare_fn(c.pfn, dev.max_smem);
            if (rc) return rc;
            int occ = 0;
            CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, c.pfn, kind->tx * kind->ty, kind->smem));
            if (occ < 1) return STENCIL_ERR_UNSUPPORTED;
            c.grid = dim3(static_cast<unsigned>(std::min<int64_t>(total, static_cast<int64_t>(dev.sms) * occ)));
            const int nt = static_cast<int>(tasks.size());
            CK(cudaMalloc(&c.dev_args, sizeof(stn::SweepArgs) * nt));
            CK(cudaMalloc(&c.dev_maps, sizeof(CUtensorMap) * nt));
            CK(cudaMalloc(&c.dev_tasks, sizeof(stn::BatchTask) * nt));
            CK(cudaMalloc(&c.dev_done, sizeof(int) * (nt + 1)));
            CK(cudaMemcpy(c.dev_args, args.data(), sizeof(stn::SweepArgs) * nt, cudaMemcpyHostToDevice));
            CK(cudaMemcpy(c.dev_maps, maps.data(), sizeof(CUtensorMap) * nt, cudaMemcpyHostToDevice));
            CK(cudaMemcpy(c.dev_tasks, tasks.data(), sizeof(stn::BatchTask) * nt, cudaMemcpyHostToDevice));
            stn::BatchArgs &B = c.args;
            B.args = static_cast<const stn::SweepArgs *>(c.dev_args);
            B.maps = static_cast<const CUtensorMap *>(c.dev_maps);
            B.tasks = static_cast<const stn::BatchTask *>(c.dev_tasks);
            B.done = static_cast<int *>(c.dev_done);
            B.head = static_cast<int *>(c.dev_done) + nt;
            B.status = dev.status;
            B.ntasks = nt;
            B.total = total;
            B.timeout_ms = timeout;
            B.fault_task = fault_task;
        }
    }
    // One CUDA graph.  Phase 0: every class resets its counters and runs its persistent launch
    // on a branch of its own, so the classes run side by side (one class's tail overlaps the
    // others' work; no class waits on another).  Phase 1, after all of phase 0: the remainder
    // passes, again one branch per class.  Captured on private streams (the caller's may be the
    // legacy stream, which cannot be captured) and launched on the caller's stream.
    (void)st;
    const int nc = static_cast<int>(E->classes.size());
    std::vector<cudaStream_t> br(nc + 1, nullptr);
    std::vector<cudaEvent_t> ev(nc + 2, nullptr);
    cudaError_t err = cudaSuccess;
    for (auto &x : br)
        if (err == cudaSuccess) err = cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking);
    for (auto &x : ev)
        if (err == cudaSuccess) err = cudaEventCreateWithFlags(&x, cudaEventDisableTiming);
    cudaGraph_t graph = nullptr;
    cudaStream_t cap = br[nc];
    if (err == cudaSuccess) err = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (err == cudaSuccess) {
        for (int phase = 0; phase < 2; ++phase) {
            // fork: every class of this phase starts after everything captured so far
            if (err == cudaSuccess) err = cudaEventRecord(ev[nc], cap);
            std::vector<int> used;
            for (int k = 0; k < nc; ++k) {
                BatchClass &c = E->classes[k];
                if (c.phase != phase) continue;
                if (err == cudaSuccess) err = cudaStreamWaitEvent(br[k], ev[nc], 0);
                if (err == cudaSuccess)
                    err = cudaMemsetAsync(c.dev_done, 0, sizeof(int) * (c.args.ntasks + 1), br[k]);
                void *args[] = {&c.args};
                if (err == cudaSuccess) err = cudaLaunchKernel(c.pfn, c.grid, c.block, args, c.smem, br[k]);
                if (err == cudaSuccess) err = cudaEventRecord(ev[k], br[k]);
                used.push_back(k);
            }
            // join
            for (int k : used)
                if (err == cudaSuccess) err = cudaStreamWaitEvent(cap, ev[k], 0);
        }
        const cudaError_t e2 = cudaStreamEndCapture(cap, &graph);
        if (err == cudaSuccess) err = e2;
    }
    if (err == cudaSuccess) err = cudaGraphInstantiate(&E->exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    for (auto x : ev)
        if (x) cudaEventDestroy(x);
    for (auto x : br)
        if (x) cudaStreamDestroy(x);
    if (err != cudaSuccess) return cuda_fail(err, __LINE__);
    return 0;
}

// ------------------------------------------------------------------------
// Scratch for stencil_run_noalloc.  Callers that must not allocate device
// memory (code inside an allocator's out-of-memory path, or processes whose
// device memory is handed out by an external budget) still need the second
// grid of the ping-pong between passes; it lives in this file-scope array
// instead, which every GPU that loads the library holds until exit.  In host
// code the array's name is only a stand-in: its device address is fetched
// once per device with cudaGetSymbolAddress below.  The status word next to it
// is where kernels launched by stencil_run_noalloc record an expired bounded
// wait; it is zero when the module loads, sticky like the main status word, and
// read and cleared by stencil_get_device_status.
constexpr size_t kNoAllocScratchBytes = size_t(16) << 20;   // 16 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];
static __device__ __align__(256) unsigned g_noalloc_status[64];

struct NoAllocDev {
    bool ready = false;
    void *scratch = nullptr;
    unsigned *status = nullptr;
    int sms = 0, max_smem = 0;
};
std::mutex g_noalloc_mu;
NoAllocDev g_noalloc[64];

// Status word of stencil_run_noalloc on device `dev`, or null if no call has set it up.
unsigned *noalloc_status_word(int dev)
{
    if (dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    return g_noalloc[dev].ready ? g_noalloc[dev].status : nullptr;
}

// Set-up of the current device (first call on that device): symbol
// addresses and the attributes the planner needs.  Allocates nothing.
int noalloc_device(NoAllocDev **out)
{
    int dev = 0;
    CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return STENCIL_ERR_NO_DEVICE;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    NoAllocDev &d = g_noalloc[dev];
    if (!d.ready) {
        CK(cudaGetSymbolAddress(&d.scratch, g_noalloc_scratch));
        void *st = nullptr;
        CK(cudaGetSymbolAddress(&st, g_noalloc_status));
        d.status = static_cast<unsigned *>(st);
        CK(cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev));
        CK(cudaDeviceGetAttribute(&d.max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
        d.ready = true;
    }
    *out = &d;
    return 0;
}

}  // namespace

extern "C" {

int stencil_create(stencil_handle *out, int dim, int radius, const float *coeffs)
{
    if (!out || !coeffs) return STENCIL_ERR_INVALID_ARG;
    *out = nullptr;
    if ((dim != 2 && dim != 3) || radius < 1 || radius > stn::kMaxR) return STENCIL_ERR_INVALID_ARG;
    stencil_plan *h = new (std::nothrow) stencil_plan;
    if (!h) return STENCIL_ERR_OOM;
    h->dim = dim;
    h->r = radius;
    h->K = 2 * dim * radius + 1;
    std::memcpy(h->c, coeffs, sizeof(float) * h->K);
    *out = h;
    return STENCIL_OK;
}

int stencil_create_shared(stencil_handle *out, int dim, int radius, const float *coeffs)
{
    if (!out || !coeffs) return STENCIL_ERR_INVALID_ARG;
    *out = nullptr;
    if ((dim != 2 && dim != 3) || radius < 1 || radius > stn::kMaxR) return STENCIL_ERR_INVALID_ARG;
    stencil_plan *h = new (std::nothrow) stencil_plan;
    if (!h) return STENCIL_ERR_OOM;
    h->dim = dim;
    h->r = radius;
    h->shared = 1;
    h->K = radius + 1;
    std::memcpy(h->c, coeffs, sizeof(float) * h->K);
    *out = h;
    return STENCIL_OK;
}

int stencil_destroy(stencil_handle h)
{
    if (!h) return STENCIL_OK;
    int rc = STENCIL_OK;
    if (h->scratch || h->dev_in || h->dev_out) {
        if (cudaDeviceSynchronize() != cudaSuccess) rc = STENCIL_ERR_CUDA;
        if (h->scratch) cudaFree(h->scratch);
        if (h->dev_in) cudaFree(h->dev_in);
        if (h->dev_out) cudaFree(h->dev_out);
    }
    delete h;
    return rc;
}

int stencil_run(stencil_handle h, const void *in, void *out, int64_t nx, int64_t ny, int64_t nz,
                int iters, int dtype, void *stream)
{
    return run_impl(h, in, out, nx, ny, nz, iters, dtype, static_cast<cudaStream_t>(stream), nullptr);
}

int stencil_run_ex(stencil_handle h, const void *in, void *out, int64_t nx, int64_t ny, int64_t nz,
                   int iters, int dtype, void *stream, const stencil_schedule *sched)
{
    return run_impl(h, in, out, nx, ny, nz, iters, dtype, static_cast<cudaStream_t>(stream), sched);
}

int stencil_run_host(stencil_handle h, const void *in_host, void *out_host, int64_t nx, int64_t ny,
                     int64_t nz, int iters, int dtype, void *stream, const stencil_schedule *sched)
{
    if (!h || !in_host || !out_host) return STENCIL_ERR_INVALID_ARG;
    int rc = check_problem(h, in_host, out_host, nx, ny, nz, iters, dtype);
    if (rc) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t bytes = static_cast<size_t>(nx * ny * nz) * elem_bytes(dtype);
    int dev = 0;
    CK(cudaGetDevice(&dev));
    if (h->host_bytes < bytes || h->host_dev != dev) {
        CK(cudaDeviceSynchronize());
        if (h->dev_in) cudaFree(h->dev_in);
        if (h->dev_out) cudaFree(h->dev_out);
        h->dev_in = h->dev_out = nullptr;
        h->host_bytes = 0;
        CK(cudaMalloc(&h->dev_in, bytes));
        CK(cudaMalloc(&h->dev_out, bytes));
        h->host_bytes = bytes;
        h->host_dev = dev;
    }
    CK(cudaMemcpyAsync(h->dev_in, in_host, bytes, cudaMemcpyHostToDevice, st));
    rc = run_impl(h, h->dev_in, h->dev_out, nx, ny, nz, iters, dtype, st, sched);
    if (rc) return rc;
    CK(cudaMemcpyAsync(out_host, h->dev_out, bytes, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return STENCIL_OK;
}

int stencil_default_schedule(stencil_handle h, int64_t nx, int64_t ny, int64_t nz, int dtype,
                             stencil_schedule *out)
{
    if (!h || !out || dtype < STENCIL_F32 || dtype > STENCIL_F16) return STENCIL_ERR_INVALID_ARG;
    chosen_schedule(h, nx, ny, nz, dtype, out);
    return STENCIL_OK;
}

int stencil_max_t(int dim, int radius, int dtype, int rows_per_thread)
{
    return registry().max_t(dim, radius, dtype, rows_per_thread, 0);
}

int stencil_get_device_status(void *stream, int clear)
{
    DevInfo *dev = nullptr;
    int rc = device_info(&dev);
    if (rc) return rc;
    int devno = 0;
    CK(cudaGetDevice(&devno));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    CK(cudaStreamSynchronize(st));
    unsigned word = 0;
    CK(cudaMemcpy(&word, dev->status, sizeof(word), cudaMemcpyDeviceToHost));
    if (clear) CK(cudaMemset(dev->status, 0, sizeof(unsigned)));
    // the word of stencil_run_noalloc's kernels on this device, once that entry point ran here
    if (unsigned *nw = noalloc_status_word(devno)) {
        unsigned w2 = 0;
        CK(cudaMemcpy(&w2, nw, sizeof(w2), cudaMemcpyDeviceToHost));
        word |= w2;
        if (clear) CK(cudaMemset(nw, 0, sizeof(unsigned)));
    }
    if (word & stn::kStatusTimeout) return STENCIL_ERR_TIMEOUT;
    if (word & stn::kStatusBounds) return STENCIL_ERR_BOUNDS;
    return STENCIL_OK;
}

int stencil_set_checked(stencil_handle h, int on)
{
    if (!h || (on != 0 && on != 1)) return STENCIL_ERR_INVALID_ARG;
    h->checked = on;
    return STENCIL_OK;
}

int stencil_set_fault_injection(stencil_handle h, int plane, int timeout_ms)
{
    if (!h) return STENCIL_ERR_INVALID_ARG;
    if (plane < 0) {
        h->fault_plane = -1;
        h->timeout_ms = 2000;
        return STENCIL_OK;
    }
    if (timeout_ms < 1 || timeout_ms > 10000) return STENCIL_ERR_INVALID_ARG;
    h->fault_plane = plane;
    h->timeout_ms = timeout_ms;
    return STENCIL_OK;
}

int stencil_run_noalloc(stencil_handle h, const void *in, void *out, int64_t nx, int64_t ny,
                        int64_t nz, int iters, int dtype, void *stream)
{
    int rc = check_problem(h, in, out, nx, ny, nz, iters, dtype);
    if (rc) return rc;
    const size_t bytes = static_cast<size_t>(nx * ny * nz) * elem_bytes(dtype);
    if (bytes > kNoAllocScratchBytes) return STENCIL_ERR_INVALID_ARG;
    NoAllocDev *nd = nullptr;
    rc = noalloc_device(&nd);
    if (rc) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // the scratch grid needs no clearing: every pass writes all of it before the next
    // pass reads it.  The status word is sticky (stencil_get_device_status clears it).
    if (iters == 0) {
        CK(cudaMemcpyAsync(out, in, bytes, cudaMemcpyDeviceToDevice, st));
        return STENCIL_OK;
    }
    DevInfo dev;
    dev.sms = nd->sms;
    dev.max_smem = nd->max_smem;
    dev.status = nd->status;
    stencil_schedule s;   // the library's rule only: no tuned or cached picks
    default_schedule(h, nx, ny, nz, dtype, &s);
    const bool aligned = (reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(out)) % 16 == 0;
    const bool streamable = s.kernel == STENCIL_KERNEL_STREAM && aligned;
    const int t = streamable ? std::max(1, std::min(s.t, iters)) : 1;
    const int L = (iters + t - 1) / t;
    const int t_last = iters - (L - 1) * t;
    Pass full, tail;
    if (streamable) {
        rc = plan_pass(h, nx, ny, nz, dtype, t, s, dev, full);
        if (rc) return rc;
        if (t_last != t) {
            rc = plan_pass(h, nx, ny, nz, dtype, t_last, s, dev, tail);
            if (rc) return rc;
        }
    }
    const void *src = in;
    for (int j = 0; j < L; ++j) {
        void *dst = ((L - 1 - j) % 2 == 0) ? out : nd->scratch;
        if (!streamable) {
            rc = launch_naive(h, src, dst, nx, ny, nz, dtype, st, dev);
            if (rc) return rc;
        } else {
            Pass &ps = (j == L - 1 && t_last != t) ? tail : full;
            ps.a.in = src;
            ps.a.out = dst;
            ps.a.status = nd->status;
            CUtensorMap map;
            std::memset(&map, 0, sizeof(map));
            if (h->dim == 3) {
                rc = encode_map(&map, src, nx, ny, nz, dtype, 4 * static_cast<int>(ps.block.x) + 2 * ps.padin,
                                static_cast<int>(ps.block.y) * s.rows_per_thread + 2 * h->r);
                if (rc) return rc;
            }
            void *args[] = {&map, &ps.a};
            CK(cudaLaunchKernel(ps.fn, ps.grid, ps.block, args, ps.smem, st));
        }
        src = dst;
    }
    return STENCIL_OK;
}

int stencil_run_batched(const stencil_batch_item *items, int n, void *stream)
{
    if (!items || n < 1) return STENCIL_ERR_INVALID_ARG;
    for (int i = 0; i < n; ++i) {
        const stencil_batch_item &b = items[i];
        int rc = check_problem(b.h, b.in, b.out, b.nx, b.ny, b.nz, b.iters, b.dtype);
        if (rc) return rc;
        if (b.iters < 1) return STENCIL_ERR_INVALID_ARG;
        const bool aligned = (reinterpret_cast<uintptr_t>(b.in) | reinterpret_cast<uintptr_t>(b.out)) % 16 == 0;
        if (!stream_applicable(b.dtype, b.nx) || !aligned) return STENCIL_ERR_UNSUPPORTED;
        const size_t bi = static_cast<size_t>(b.nx * b.ny * b.nz) * elem_bytes(b.dtype);
        for (int j = 0; j < n; ++j) {   // no input or output may overlap another item's output
            if (j == i) continue;
            const stencil_batch_item &c = items[j];
            const size_t bj = static_cast<size_t>(c.nx * c.ny * c.nz) * elem_bytes(c.dtype);
            if (ranges_overlap(b.out, bi, c.out, bj) || ranges_overlap(b.in, bi, c.out, bj))
                return STENCIL_ERR_ALIAS;
        }
    }
    DevInfo *dev = nullptr;
    int rc = device_info(&dev);
    if (rc) return rc;
    int devno = 0;
    CK(cudaGetDevice(&devno));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    std::lock_guard<std::mutex> lk(g_batch_mu);
    const std::vector<char> key = batch_key(items, n, devno);
    BatchEntry *E = nullptr;
    for (size_t i = 0; i < g_batch.size(); ++i)
        if (g_batch[i]->key == key) {
            E = g_batch[i];
            g_batch.erase(g_batch.begin() + static_cast<long>(i));
            g_batch.push_back(E);
            break;
        }
    if (!E) {
        E = new (std::nothrow) BatchEntry;
        if (!E) return STENCIL_ERR_OOM;
        E->key = key;
        E->dev = devno;
        rc = build_batch(items, n, *dev, st, E);
        if (rc) {
            free_entry(E);
            return rc;
        }
        g_batch.push_back(E);
        while (g_batch.size() > 4) {
            free_entry(g_batch.front());
            g_batch.erase(g_batch.begin());
        }
    }
    CK(cudaGraphLaunch(E->exec, st));
    return STENCIL_OK;
}

int stencil_resolve_schedule(stencil_handle h, int64_t nx, int64_t ny, int64_t nz, int dtype,
                             const stencil_schedule *sched, stencil_schedule *out)
{
    if (!h || !out || nx <= 0 || ny <= 0 || nz <= 0 || (h->dim == 2 && nz != 1) || dtype < STENCIL_F32 ||
        dtype > STENCIL_F16)
        return STENCIL_ERR_INVALID_ARG;
    DevInfo *dev = nullptr;
    int rc = device_info(&dev);
    if (rc) return rc;
    stencil_schedule s;
    chosen_schedule(h, nx, ny, nz, dtype, &s);
    if (sched) {
        if (sched->t) s.t = sched->t;
        if (sched->rows_per_thread) s.rows_per_thread = sched->rows_per_thread;
        if (sched->seg) s.seg = sched->seg;
        if (sched->threads_x) s.threads_x = sched->threads_x;
        if (sched->threads_y) s.threads_y = sched->threads_y;
        if (sched->planes_per_step) s.planes_per_step = sched->planes_per_step;
        if (sched->prefetch) s.prefetch = sched->prefetch;
    }
    if (!stream_applicable(dtype, nx) || s.t < 1) return STENCIL_ERR_UNSUPPORTED;
    Pass ps;
    return resolve(h, nx, ny, nz, dtype, s, *dev, *out, ps);
}

int stencil_schedule_features(stencil_handle h, int64_t nx, int64_t ny, int64_t nz, int dtype,
                              const stencil_schedule *sched, float *features)
{
    if (!h || !features || nx <= 0 || ny <= 0 || nz <= 0 || dtype < STENCIL_F32 || dtype > STENCIL_F16)
        return STENCIL_ERR_INVALID_ARG;
    DevInfo *dev = nullptr;
    int rc = device_info(&dev);
    if (rc) return rc;
    stencil_schedule s;
    default_schedule(h, nx, ny, nz, dtype, &s);
    if (sched) {
        if (sched->t) s.t = sched->t;
        if (sched->rows_per_thread) s.rows_per_thread = sched->rows_per_thread;
        if (sched->seg) s.seg = sched->seg;
        if (sched->threads_x) s.threads_x = sched->threads_x;
        if (sched->threads_y) s.threads_y = sched->threads_y;
        if (sched->planes_per_step) s.planes_per_step = sched->planes_per_step;
    }
    stencil_schedule r;
    Pass ps;
    rc = resolve(h, nx, ny, nz, dtype, s, *dev, r, ps);
    if (rc) return rc;
    features_of(h, nx, ny, nz, dtype, r, ps, analytic_ns(h, nx, ny, nz, dtype, r, ps.occ, dev->sms), dev->sms, features);
    return STENCIL_OK;
}

int stencil_tune(stencil_handle h, int64_t nx, int64_t ny, int64_t nz, int dtype, int mode,
                 stencil_model_handle model, int store, stencil_schedule *chosen, stencil_timing *rows,
                 int cap, int *nrows)
{
    if (!h || !chosen || nx <= 0 || ny <= 0 || nz <= 0 || (h->dim == 2 && nz != 1) || dtype < STENCIL_F32 ||
        dtype > STENCIL_F16 || mode < STENCIL_TUNE_ANALYTIC || mode > STENCIL_TUNE_MODEL ||
        (mode == STENCIL_TUNE_MODEL && !model) || (rows && cap < 0))
        return STENCIL_ERR_INVALID_ARG;
    if (!stream_applicable(dtype, nx)) return STENCIL_ERR_UNSUPPORTED;
    DevInfo *dev = nullptr;
    int rc = device_info(&dev);
    if (rc) return rc;
    stencil_schedule cand[512];
    const int nc0 = candidates(h, ny, nz, dtype, cand, 512);
    std::vector<stencil_timing> tim;
    std::vector<Pass> passes;
    for (int i = 0; i < nc0; ++i) {
        stencil_schedule r;
        Pass ps;
        if (resolve(h, nx, ny, nz, dtype, cand[i], *dev, r, ps)) continue;   // tile too small etc.
        bool dup = false;   // several requested segment lengths can resolve to the same one
        for (const auto &x : tim)
            if (x.sched.t == r.t && x.sched.seg == r.seg && x.sched.rows_per_thread == r.rows_per_thread &&
                x.sched.planes_per_step == r.planes_per_step)
                dup = true;
        if (dup) continue;
        stencil_timing tm{};
        tm.sched = r;
        tm.analytic_ns_per_cell = static_cast<float>(analytic_ns(h, nx, ny, nz, dtype, r, ps.occ, dev->sms));
        features_of(h, nx, ny, nz, dtype, r, ps, tm.analytic_ns_per_cell, dev->sms, tm.features);
        tm.ns_per_cell = -1.f;
        tm.model_ns_per_cell = -1.f;
        tim.push_back(tm);
    }
    if (tim.empty()) return STENCIL_ERR_UNSUPPORTED;
    const int nc = static_cast<int>(tim.size());
    if (mode == STENCIL_TUNE_MODEL) {
        std::vector<float> X(static_cast<size_t>(nc) * STENCIL_NFEAT), y(nc);
        for (int i = 0; i < nc; ++i) std::memcpy(&X[static_cast<size_t>(i) * STENCIL_NFEAT], tim[i].features, sizeof(tim[i].features));
        rc = stencil_model_predict(model, X.data(), y.data(), nc);
        if (rc) return rc;
        // the model predicts the log of measured over analytic time
        for (int i = 0; i < nc; ++i) tim[i].model_ns_per_cell = tim[i].analytic_ns_per_cell * std::exp(y[i]);
    }
    if (mode == STENCIL_TUNE_EXHAUSTIVE) {
        const size_t bytes = static_cast<size_t>(nx * ny * nz) * elem_bytes(dtype);
        void *a = nullptr, *b = nullptr;
        CK(cudaMalloc(&a, bytes));
        if (cudaMalloc(&b, bytes) != cudaSuccess) {
            cudaFree(a);
            return STENCIL_ERR_OOM;
        }
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        cudaMemset(a, 0, bytes);
        int err = 0;
        // every timing covers >= 16 steps and, for small grids, >= 2^30 cell updates (about a
        // millisecond): shorter runs are dominated by launch latency and jitter
        const double cells = static_cast<double>(nx) * ny * nz;
        const int steps = static_cast<int>(std::min(1000.0, std::max(16.0, std::ceil(1073741824.0 / cells))));
        for (int i = 0; i < nc && !err; ++i) {
            const int t = tim[i].sched.t;
            const int iters = t * std::max(2, (steps + t - 1) / t);
            err = run_impl(h, a, b, nx, ny, nz, iters, dtype, nullptr, &tim[i].sched);
            float best = 1e30f;
            for (int rep = 0; rep < 2 && !err; ++rep) {
                cudaEventRecord(e0, nullptr);
                err = run_impl(h, a, b, nx, ny, nz, iters, dtype, nullptr, &tim[i].sched);
                cudaEventRecord(e1, nullptr);
                if (cudaEventSynchronize(e1) != cudaSuccess) err = STENCIL_ERR_CUDA;
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                best = std::min(best, ms);
            }
            tim[i].ns_per_cell = static_cast<float>(best * 1e6 / (static_cast<double>(nx) * ny * nz * iters));
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        cudaFree(a);
        cudaFree(b);
        if (err) return err;
    }
    int best = 0;
    auto key = [&](const stencil_timing &x) {
        return mode == STENCIL_TUNE_EXHAUSTIVE ? x.ns_per_cell
               : mode == STENCIL_TUNE_MODEL   ? x.model_ns_per_cell
                                              : x.analytic_ns_per_cell;
    };
    for (int i = 1; i < nc; ++i)
        if (key(tim[i]) < key(tim[best])) best = i;
    if (mode == STENCIL_TUNE_MODEL) {
        // trust region around the analytic pick: the learned correction replaces it only where
        // it predicts at least kModelMargin less time for its own pick than for the analytic one
        // (smaller predicted gains are within the model's fit error, log-RMS about 7 %)
        int ia = 0;
        for (int i = 1; i < nc; ++i)
            if (tim[i].analytic_ns_per_cell < tim[ia].analytic_ns_per_cell) ia = i;
        constexpr float kModelMargin = 0.05f;
        if (!(tim[best].model_ns_per_cell < (1.f - kModelMargin) * tim[ia].model_ns_per_cell)) best = ia;
    }
    *chosen = tim[best].sched;
    if (store) {
        bool found = false;
        for (auto &tu : h->tuned)
            if (tu.nx == nx && tu.ny == ny && tu.nz == nz && tu.dtype == dtype) {
                tu.s = *chosen;
                found = true;
            }
        if (!found) h->tuned.push_back({nx, ny, nz, dtype, *chosen});
        fc_store(h, nx, ny, nz, dtype, *chosen);
    }
    if (rows)
        for (int i = 0; i < nc && i < cap; ++i) rows[i] = tim[i];
    if (nrows) *nrows = nc;
    return STENCIL_OK;
}

int stencil_use_cost_model(stencil_model_handle m)
{
    std::lock_guard<std::mutex> lk(g_model_mu);
    g_model = m;
    ++g_model_gen;
    return STENCIL_OK;
}

int stencil_last_cuda_error(void) { return g_last_cuda_error; }

const char *stencil_strerror(int code)
{
    switch (code) {
    case STENCIL_OK: return "ok";
    case STENCIL_ERR_INVALID_ARG: return "invalid argument";
    case STENCIL_ERR_ALIAS: return "input and output overlap";
    case STENCIL_ERR_UNSUPPORTED: return "schedule not supported for this problem";
    case STENCIL_ERR_OOM: return "device allocation failed";
    case STENCIL_ERR_CUDA: return "CUDA call failed";
    case STENCIL_ERR_TIMEOUT: return "kernel bounded wait expired";
    case STENCIL_ERR_NO_DEVICE: return "no usable GPU";
    case STENCIL_ERR_BOUNDS: return "bounds-checked kernel found an out-of-range access";
    default: return "unknown status";
    }
}

}  // extern "C"
