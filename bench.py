"""Benchmark: repeated 2D star-stencil sweeps, radius 1..4, 16384 x 16384 FP32 grid,
1000 iterations per radius, clamp to edge, each radius at the library's chosen
temporal degree.  One "step" = the four radii back to back (4 x 1000 sweeps of
the 1 GiB grid).  Metric: GCell/s = cells * iterations / time (Section IV.C,
Eq. 3 of the paper), whole job over all ranks.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the CPU oracle (the plain C sweep, OpenMP over the
host cores) on a bounded crop of the same workload; it is the baseline the
GPU path is compared with, and the only other place this file runs the oracle
is the cpu_baseline field of the GPU line.
Under torchrun (N > 1) every rank sweeps its own grids (independent problems,
weak scaling, no collective on the data path); the barrier and a max-reduce
of the elapsed time use the process group.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import platform
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import stencil_inputs as gen  # noqa: E402

METRIC = "GCell/s & GFLOP/s per radius (2D/3D), plain FP32 vs tuned/BF16, % of roofline"
NX = NY = 16384
ITERS = 1000
RADII = (1, 2, 3, 4)
WORKLOAD = "2D star stencils r=1..4, 16384x16384 FP32, 1000 iterations each, clamp to edge"
SAMPLE_SIDE = 2048          # oracle sample: top-left 2048x2048 crop of the same input
SAMPLE_ITERS = 100
FALLBACK_HBM_GBS = 6800.0


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def crop_input(side: int) -> np.ndarray:
    """Top-left side x side crop of the seeded 16384^2 input (same counters)."""
    out = np.empty((side, side), np.float32)
    for y in range(side):
        gen.uniform(gen.GRID_SEED, side, offset=y * NX, out=out[y])
    return out


def peaks(measure: bool = True):
    """Roofline denominators: HBM from MEASURED_PEAKS.json (the pool's copy measurement), FP32
    from the library's FMA-throughput kernel on this device (nominal unit count x clock if not
    measured)."""
    p = {"hbm_gbs": FALLBACK_HBM_GBS, "hbm_src": "fallback"}
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            m = json.load(fh)
        if m.get("hbm_gbs"):
            p = {"hbm_gbs": float(m["hbm_gbs"]), "hbm_src": "measured"}
    from paper_2002_05983_gb300 import metrics
    p["fp32_flops"] = metrics.FP32_PEAK_NOMINAL
    p["fp32_src"] = "nominal: 152 SMs x 128 FP32 lanes x 2 FLOP x 2070 MHz"
    if measure:
        import paper_2002_05983_gb300 as st
        m = st.stencil_measure_peaks()
        p["fp32_flops"] = m.fp32_flops
        p["fp32_src"] = (f"measured: FMA-throughput kernel, {m.sms} SMs "
                         f"(nominal {metrics.FP32_PEAK_NOMINAL / 1e12:.2f} TFLOP/s)")
        p["copy_gbs_library"] = m.copy_bytes_per_s / 1e9
    return p


class Clocks:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        sm, mx, reasons = [], None, set()
        for ln in getattr(self, "lines", []):
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0]))
                mx = float(f[1])
            except ValueError:
                continue
            for n, v in zip(names, f[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        out = {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
               "samples": len(sm)}
        watts = []
        for ln in getattr(self, "lines", []):
            try:
                watts.append(float(ln.split(",")[2]))
            except (IndexError, ValueError):
                pass
        if watts:
            out["power_w"] = round(statistics.median(watts), 1)
        return out


def parse_cpulist(text: str):
    """'0-3,8,10-11' -> {0, 1, 2, 3, 8, 10, 11}; None if it is not a CPU list."""
    cpus = set()
    for part in text.strip().split(","):
        lo, _, hi = part.partition("-")
        if not lo.isdigit() or (hi and not hi.isdigit()):
            return None
        cpus.update(range(int(lo), int(hi or lo) + 1))
    return cpus or None


def gpu_local_cpus(index: int):
    """CPUs next to GPU `index` (nvidia-smi topo's CPU affinity), or None if unknown."""
    try:
        out = subprocess.run(["nvidia-smi", "topo", "-m"], capture_output=True, text=True, timeout=30).stdout
    except (OSError, subprocess.TimeoutExpired):
        return None
    lines = [ln for ln in out.splitlines() if ln.strip()]
    head = next((ln for ln in lines if "CPU Affinity" in ln), None)
    row = next((ln for ln in lines if ln is not head and ln.split() and ln.split()[0] == f"GPU{index}"), None)
    if not head or not row:
        return None
    cols = [c.strip() for c in head.split("\t")]
    if cols and not cols[0]:
        cols = cols[1:]                   # the header has no row-label column
    vals = [c.strip() for c in row.split("\t")]
    if "CPU Affinity" not in cols or len(vals) < len(cols) + 1:
        return None
    cpus = parse_cpulist(vals[cols.index("CPU Affinity") + 1])
    return cpus & os.sched_getaffinity(0) if cpus else None


# ---- replicas (one process per GPU, weak scaling): rank environment and timing reduction
def rank_env():
    """(world, rank, local rank) from the torchrun environment (1, 0, 0 without it)."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def reduce_max(value: float, dist=None, device="cpu") -> float:
    """Largest `value` over all ranks (the job's time is its slowest rank's)."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: float, world: int, seconds: float) -> float:
    """Whole-job throughput: every rank processed units_per_rank in at most `seconds`."""
    return units_per_rank * world / seconds


def kernel_source_hash(csrc):
    """sha256[:16] of the streaming kernel's sources (kernel body, then tile geometry)."""
    h = hashlib.sha256()
    for name in ("sweep_kernel.cuh", "sweep_cfg.h"):
        with open(os.path.join(csrc, name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def traffic_for(dim, r, t, dtype="f32"):
    """DRAM bytes per launch from the committed ncu summary, if the kernel source is unchanged."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    csrc = os.path.join(ROOT, "paper_2002_05983_gb300", "csrc")
    if not os.path.exists(path):
        return None
    h = kernel_source_hash(csrc)
    for ln in open(path):
        f = ln.split()
        if len(f) == 6 and not ln.startswith("#") and f[0] == h and f[1:5] == [str(dim), str(r), str(t), dtype]:
            return int(f[5])
    return None


def limiter_for(dim, r, t, hbm_frac, dtype="f32"):
    """What limits a kernel: ncu's DRAM / FMA-pipe / issue figures from the committed summary (while
    the kernel sources keep that hash) and the live fraction of the HBM roof.  "hbm" when the live
    bandwidth is >= 85 % of the measured copy peak or ncu shows DRAM >= 80 %, "alu" when the FMA pipe
    is >= 80 % busy, else "issue" (neither unit saturated: the issue rate and latencies set the speed)."""
    path = os.path.join(ROOT, "profiles", "ncu_limits.txt")
    csrc = os.path.join(ROOT, "paper_2002_05983_gb300", "csrc")
    out = {"hbm_frac_live": round(hbm_frac, 4) if hbm_frac is not None else None}
    if os.path.exists(path):
        h = kernel_source_hash(csrc)
        for ln in open(path):
            f = ln.split()
            if len(f) == 10 and not ln.startswith("#") and f[0] == h and f[1:5] == [str(dim), str(r), str(t), dtype]:
                out.update(dram_pct=float(f[5]), fma_pipe_pct=float(f[6]), issue_per_scheduler=float(f[7]),
                           top_stall=f[8], source="ncu, profiles/ncu_limits.txt")
    if (hbm_frac or 0) >= 0.85 or out.get("dram_pct", 0) >= 80:
        out["kind"] = "hbm"
    elif out.get("fma_pipe_pct", 0) >= 80:
        out["kind"] = "alu"
    elif "dram_pct" in out:
        out["kind"] = "issue"
    else:
        out["kind"] = None   # no counters for this kernel source
    return out


def host_cpu():
    """CPU model (from /proc/cpuinfo, else the machine type) and the CPUs this process may use."""
    model = platform.machine()
    try:
        with open("/proc/cpuinfo") as fh:
            for ln in fh:
                key = ln.split(":")[0].strip().lower()
                if key in ("model name", "cpu model", "hardware"):
                    model = ln.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    return {"model": model, "cpus_allowed": len(os.sched_getaffinity(0))}


def oracle_leg(steps: int, warmup: int):
    """Time the CPU oracle on the crop; returns (GCell/s, seconds per step, cores, sample text)."""
    import oracle
    oracle.build()
    f = crop_input(SAMPLE_SIDE)
    coeffs = {r: gen.coefficients(2, r) for r in RADII}
    cores = oracle.max_threads()

    def one():
        for r in RADII:
            oracle.sweep_f32(f, 2, r, coeffs[r], SAMPLE_ITERS)

    for _ in range(warmup):
        one()
    t0 = time.perf_counter()
    for _ in range(steps):
        one()
    dt = (time.perf_counter() - t0) / steps
    cells = SAMPLE_SIDE * SAMPLE_SIDE * SAMPLE_ITERS * len(RADII)
    sample = (f"oracle_sweep_f32 on the top-left {SAMPLE_SIDE}x{SAMPLE_SIDE} crop of the same input, "
              f"r=1..4, {SAMPLE_ITERS} iterations each")
    return cells / dt / 1e9, dt, cores, sample


def reference_main(args):
    _, rank, _ = rank_env()
    if rank != 0:   # the oracle arm runs once, on rank 0; other ranks exit without work
        return 0
    g, dt, cores, sample = oracle_leg(args.steps, args.warmup)
    line = {"impl": "reference", "metric": METRIC, "value": round(g, 4), "unit": "GCell/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(dt * 1e3, 3), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": sample, "l2": "n/a (host)"},
            "cpu_baseline": {"value": round(g, 4), "unit": "GCell/s", "cores": cores, "kind": "oracle",
                             "sample": sample, "cpu": host_cpu()},
            "e2e": {"value": round(g, 4), "unit": "GCell/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def case_main(args):
    """One radius on an n^dim grid: the small case used for ncu captures."""
    import torch
    import paper_2002_05983_gb300 as st
    f = args.case.split(":")
    dim, r, t, n, iters = (int(v) for v in f[:5])
    dt = f[5] if len(f) > 5 else "f32"
    pps = int(f[6]) if len(f) > 6 else 0          # 2D rows per step (0: the library's choice)
    tdt = {"f32": torch.float32, "bf16": torch.bfloat16, "f16": torch.float16}[dt]
    shape = (n, n) if dim == 2 else (n, n, n)
    x = torch.from_numpy(gen.workload_grid(dim, *shape[::-1])).to(tdt).cuda()
    out = torch.empty_like(x)
    s = st.Stencil(dim, r, gen.coefficients(dim, r))
    sched = st.schedule(kernel=st.KERNEL_STREAM, t=t, planes_per_step=pps) if t else None
    for _ in range(args.warmup):
        s.run(x, iters, out=out, sched=sched)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        s.run(x, iters, out=out, sched=sched)
    e1.record()
    torch.cuda.synchronize()
    sec = e0.elapsed_time(e1) / 1e3 / args.steps
    assert st.stencil_get_device_status() == 0
    print(json.dumps({"case": args.case, "gcells": round(x.numel() * iters / sec / 1e9, 2),
                      "ms": round(sec * 1e3, 3)}), flush=True)
    return 0


def _timed(fn, reps=2):
    import torch
    fn()
    torch.cuda.synchronize()
    best = 1e30
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1) / 1e3)
    return best


def _rand(shape, dtype, seed):
    import torch
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    return torch.rand(shape, device="cuda", generator=g).to(dtype)


def _row(**kw):
    print(json.dumps(kw), flush=True)


def suite_main(args):
    """Measurements of the other workloads.  Timing grids are torch.rand on the device (values do
    not change the speed); parity and error figures use the seeded workload inputs."""
    import torch
    import oracle
    import paper_2002_05983_gb300 as st
    from paper_2002_05983_gb300 import metrics
    torch.cuda.set_device(0)
    pk = peaks()
    f32 = torch.float32

    def roof(dim, r, t, es):
        return metrics.roofline_cells(dim, r, t, es, pk["fp32_flops"], pk["hbm_gbs"] * 1e9) / 1e9

    if args.suite in ("sweep2d", "sweep3d"):
        dim = 2 if args.suite == "sweep2d" else 3
        shape, iters = ((16384, 16384), 1000) if dim == 2 else ((512, 512, 512), 200)
        x = _rand(shape, f32, 0)
        out = torch.empty_like(x)
        n = x.numel()
        radii = [int(v) for v in args.radii.split(",")]
        for r in radii:
            s = st.Stencil(dim, r, gen.coefficients(dim, r))
            for vy in ((1,) if dim == 2 else (2, 4)):
                for t in range(1, st.stencil_max_t(dim, r, 0, vy) + 1):
                    for pps in ((1, 2, 4) if dim == 2 else (1,)):
                        sc = st.schedule(kernel=st.KERNEL_STREAM, t=t, rows_per_thread=vy, planes_per_step=pps)
                        try:
                            res = st.stencil_resolve_schedule(s.handle, *(shape[::-1] + ((1,) if dim == 2 else ())),
                                                              st.STENCIL_F32, sc)
                        except st.StencilError:
                            continue
                        if res.planes_per_step != pps:
                            continue   # no kernel with this many rows per step at this degree
                        sec = _timed(lambda: s.run(x, iters, out=out, sched=sc), reps=1)
                        g = n * iters / sec / 1e9
                        _row(suite=args.suite, dim=dim, r=r, t=t, rows_per_thread=vy, planes_per_step=pps,
                             iters=iters, grid=list(shape), gcells=round(g, 1),
                             gflops=round(g * metrics.flop_per_cell(dim, r), 1),
                             roofline_gcells=round(roof(dim, r, t, 4), 1), roofline_frac=round(g / roof(dim, r, t, 4), 4))
            sec = _timed(lambda: s.run(x, iters, out=out), reps=1)
            d = s.default_schedule(shape)
            _row(suite=args.suite, dim=dim, r=r, default_t=d.t, default_rows=d.rows_per_thread,
                 default_planes_per_step=d.planes_per_step, gcells_default=round(n * iters / sec / 1e9, 1))
        # parity on the seeded crop at the full step count (clamp at the crop's own edges)
        side = 1024 if dim == 2 else 128
        f = crop_input(side) if dim == 2 else gen.workload_grid(3, side, side, side)
        for r in radii:
            c = gen.coefficients(dim, r)
            s = st.Stencil(dim, r, c)
            got = s.run(torch.from_numpy(f).cuda(), iters).cpu().numpy()
            w32 = oracle.sweep_f32(f, dim, r, c, iters)
            w64 = oracle.sweep_f64(f.astype(np.float64), dim, r, c.astype(np.float64), iters)
            _row(suite=args.suite, parity=True, dim=dim, r=r, crop=side, iters=iters,
                 bit_exact_vs_fp32_oracle=bool(np.array_equal(got, w32)),
                 max_abs_vs_fp64=float(np.max(np.abs(got - w64))), bound=2e-6 * iters)
        return 0

    if args.suite == "shared":
        # one coefficient per distance vs one per (distance, direction), default schedules
        for dim, shape, iters, side in ((2, (16384, 16384), 1000, 1024), (3, (512, 512, 512), 200, 128)):
            x = _rand(shape, f32, 0)
            out = torch.empty_like(x)
            n = x.numel()
            for r in RADII:
                full = st.Stencil(dim, r, gen.coefficients(dim, r))
                sh = st.Stencil(dim, r, gen.shared_coefficients(dim, r), shared=True)
                g_full = n * iters / _timed(lambda: full.run(x, iters, out=out), reps=1) / 1e9
                g_sh = n * iters / _timed(lambda: sh.run(x, iters, out=out), reps=1) / 1e9
                f_sh = 1 + r * (2 * dim + 1)   # FLOP per cell update with shared coefficients
                _row(suite="shared", dim=dim, r=r, grid=list(shape), iters=iters, t=sh.default_schedule(shape).t,
                     gcells_shared=round(g_sh, 1), gflops_shared=round(g_sh * f_sh, 1), flop_per_cell_shared=f_sh,
                     gcells_full=round(g_full, 1), gflops_full=round(g_full * metrics.flop_per_cell(dim, r), 1))
            del x, out
            f = crop_input(side) if dim == 2 else gen.workload_grid(3, side, side, side)
            for r in RADII:
                c = gen.shared_coefficients(dim, r)
                got = st.Stencil(dim, r, c, shared=True).run(torch.from_numpy(f).cuda(), iters).cpu().numpy()
                w32 = oracle.sweep_shared_f32(f, dim, r, c, iters)
                w64 = oracle.sweep_shared_f64(f.astype(np.float64), dim, r, c.astype(np.float64), iters)
                _row(suite="shared", parity=True, dim=dim, r=r, crop=side, iters=iters,
                     bit_exact_vs_fp32_oracle=bool(np.array_equal(got, w32)),
                     max_abs_vs_fp64=float(np.max(np.abs(got - w64))), bound=2e-6 * iters)
        return 0

    if args.suite == "precision":
        iters = 500
        for dim, shape, small in ((3, (768, 768, 768), 128), (2, (32768, 32768), 2048)):
            r = 4
            s = st.Stencil(dim, r, gen.coefficients(dim, r))
            base = None
            for name, dt, es in (("f32", torch.float32, 4), ("bf16", torch.bfloat16, 2), ("f16", torch.float16, 2)):
                x = _rand(shape, dt, 1)
                out = torch.empty_like(x)
                sec = _timed(lambda: s.run(x, iters, out=out), reps=1)
                g = x.numel() * iters / sec / 1e9
                base = base or g
                t = s.default_schedule(shape, st.dtype_code(x)).t
                _row(suite="precision", dim=dim, r=r, dtype=name, grid=list(shape), iters=iters, t=t,
                     gcells=round(g, 1), speedup_vs_f32=round(g / base, 3),
                     roofline_frac=round(g / roof(dim, r, t, es), 4))
                del x, out
                torch.cuda.empty_cache()
            # accuracy on the small instance, 500 steps, against the FP64 oracle
            f = gen.workload_grid(dim, *((small,) * dim))
            c = gen.coefficients(dim, r)
            w64 = oracle.sweep_f64(f.astype(np.float64), dim, r, c.astype(np.float64), iters)
            for name, dt in (("f32", torch.float32), ("bf16", torch.bfloat16), ("f16", torch.float16)):
                xs = torch.from_numpy(f).to(dt)
                got = s.run(xs.cuda(), iters).float().cpu().numpy().astype(np.float64)
                w_in = oracle.sweep_f64(xs.float().numpy().astype(np.float64), dim, r, c.astype(np.float64), iters)
                _row(suite="precision", accuracy=True, dim=dim, r=r, dtype=name, grid=[small] * dim, iters=iters,
                     max_abs=float(np.max(np.abs(got - w64))),
                     rel_l2=float(np.linalg.norm(got - w64) / np.linalg.norm(w64)),
                     max_abs_vs_rounded_input=float(np.max(np.abs(got - w_in))),
                     rel_l2_vs_rounded_input=float(np.linalg.norm(got - w_in) / np.linalg.norm(w_in)))
        return 0

    if args.suite == "batch":
        iters = 100
        items = gen.batch_list()
        for it in items:   # rows must be 16-byte aligned for the streaming kernel
            it["nx"] -= it["nx"] % 8
        stencils, bufs, batch = {}, [], []
        for k, it in enumerate(items):
            key = (it["dim"], it["r"])
            if key not in stencils:
                stencils[key] = st.Stencil(it["dim"], it["r"], gen.coefficients(*key))
            shape = (it["ny"], it["nx"]) if it["dim"] == 2 else (it["nz"], it["ny"], it["nx"])
            dt = torch.bfloat16 if it["dtype"] == "bf16" else torch.float32
            x = _rand(shape, dt, 100 + k)
            y = torch.empty_like(x)
            bufs.append((x, y))
            batch.append((stencils[key].handle, x.data_ptr(), y.data_ptr(), it["nx"], it["ny"], it["nz"], iters,
                          st.dtype_code(x)))
        stream = torch.cuda.current_stream().cuda_stream
        cells = sum(b[3] * b[4] * b[5] for b in batch) * iters

        def singles():
            for (h, xp, yp, nx, ny, nz, it_, code), (x, y) in zip(batch, bufs):
                st.stencil_run(h, xp, yp, nx, ny, nz, it_, code, stream)

        t_single = _timed(singles, reps=2)
        ref = [y.clone() for _, y in bufs]
        t_batch = _timed(lambda: st.stencil_run_batched(batch, stream), reps=3)
        assert st.stencil_get_device_status() == 0
        same = sum(int(torch.equal(y, r)) for (x, y), r, it in zip(bufs, ref, items) if it["dtype"] == "f32")
        n32 = sum(1 for it in items if it["dtype"] == "f32")
        _row(suite="batch", grids=len(batch), grids_2d=sum(1 for it in items if it["dim"] == 2), iters=iters,
             cell_updates=cells, seconds_individual=round(t_single, 4), seconds_batched=round(t_batch, 4),
             gcells_individual=round(cells / t_single / 1e9, 1), gcells_batched=round(cells / t_batch / 1e9, 1),
             speedup=round(t_single / t_batch, 3), fp32_grids_bit_identical_to_individual=f"{same}/{n32}")
        return 0
    return 1


def tune_main(args):
    """Tuner evaluation: >= 2000 measured schedule timings on seeded problems shaped like the
    batched workload, cost model trained on 64 problems, regret on 16 held-out ones."""
    import torch
    from paper_2002_05983_gb300 import tune
    torch.cuda.set_device(0)
    t0 = time.time()
    res = tune.evaluate(n_train=64, n_test=16, seed=3, epochs=4000)

    def stats(rows, key):
        v = np.array([r[key] for r in rows], np.float64)
        return {"mean": round(float(np.nanmean(v)), 4), "median": round(float(np.nanmedian(v)), 4),
                "max": round(float(np.nanmax(v)), 4), "within_10pct": int(np.sum(v <= 0.10)), "n": int(len(v))}

    out = {"tune_eval": True, "rows_total": res["rows_total"], "rows_train": res["rows_train"],
           "train_loss": round(res["train_loss"], 5), "seconds": round(time.time() - t0, 1),
           "regret_model_test": stats(res["test"], "regret_model"),
           "regret_analytic_test": stats(res["test"], "regret_analytic"),
           "regret_model_train": stats(res["train"], "regret_model"),
           "analytic_model_accuracy": {
               "measured_over_predicted_median": round(float(np.median(res["analytic_ratio"])), 3),
               "p10": round(float(np.percentile(res["analytic_ratio"], 10)), 3),
               "p90": round(float(np.percentile(res["analytic_ratio"], 90)), 3),
               "rows": int(len(res["analytic_ratio"]))},
           "test_problems": [dict(r["problem"], best_ns=round(r["best_ns"], 5),
                                  regret_model=round(r["regret_model"], 4),
                                  regret_analytic=round(r["regret_analytic"], 4)) for r in res["test"]]}
    print(json.dumps(out), flush=True)
    return 0


def _event_time(fn, reps, stream):
    """Best CUDA-event time of fn() on `stream` over reps runs (after one warm-up run)."""
    import torch
    fn()
    torch.cuda.synchronize()
    best = 1e30
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1) / 1e3)
    return best


def measure_3d(pk, stream):
    """3D 512^3 FP32, 200 iterations, radius 1..4 at the library's default schedule (seeded
    uniform + Gaussian-bump input); per radius GCell/s and the fraction of R(t)."""
    import torch
    import paper_2002_05983_gb300 as st
    from paper_2002_05983_gb300 import metrics
    n, iters = 512, 200
    x = torch.from_numpy(gen.workload_grid(3, n, n, n)).cuda()
    out = torch.empty_like(x)
    rows = []
    for r in RADII:
        s = st.Stencil(3, r, gen.coefficients(3, r))
        d = s.default_schedule((n, n, n))
        sec = _event_time(lambda: s.run(x, iters, out=out), 3, stream)
        g = x.numel() * iters / sec / 1e9
        roof = metrics.roofline_cells(3, r, d.t, 4, pk["fp32_flops"], pk["hbm_gbs"] * 1e9) / 1e9
        rows.append({"r": r, "t": d.t, "rows_per_thread": d.rows_per_thread, "gcells": round(g, 2),
                     "gflops": round(g * metrics.flop_per_cell(3, r), 1), "roofline_gcells": round(roof, 1),
                     "roofline_frac": round(g / roof, 4),
                     "bound": metrics.roofline_bound(3, r, d.t, 4, pk["fp32_flops"], pk["hbm_gbs"] * 1e9),
                     "limiter": limiter_for(3, r, d.t, g * 8 / (d.t * pk["hbm_gbs"])),
                     "ms": round(sec * 1e3, 2)})
        s.close()
    assert st.stencil_get_device_status() == 0
    return {"grid": [n, n, n], "iters": iters, "input": "uniform [0,1) seed 0 + Gaussian bump sigma 16",
            "radii": rows}


def measure_precision(pk, stream):
    """Radius 4 on 768^3 (3D) and 32768^2 (2D), 500 iterations, FP32 vs BF16 vs FP16 storage at the
    default schedules: speed-up over FP32 (timing grids: torch.rand on the device, values do not
    change the speed), and the error after 500 steps against the FP64 oracle on the seeded
    128^3 / 2048^2 instances."""
    import torch
    import oracle
    import paper_2002_05983_gb300 as st
    from paper_2002_05983_gb300 import metrics
    iters, r = 500, 4
    out = {}
    dts = (("f32", torch.float32, 4), ("bf16", torch.bfloat16, 2), ("f16", torch.float16, 2))
    for dim, n, small in ((3, 768, 128), (2, 32768, 2048)):
        s = st.Stencil(dim, r, gen.coefficients(dim, r))
        key = f"{dim}d_{n}"
        res = {}
        g = torch.Generator(device="cuda")
        g.manual_seed(1)
        for name, dt, es in dts:
            x = torch.rand((n,) * dim, device="cuda", generator=g).to(dt)
            y = torch.empty_like(x)
            d = s.default_schedule((n,) * dim, st.dtype_code(x))
            sec = _event_time(lambda: s.run(x, iters, out=y), 1, stream)
            gc = x.numel() * iters / sec / 1e9
            roof = metrics.roofline_cells(dim, r, d.t, es, pk["fp32_flops"], pk["hbm_gbs"] * 1e9) / 1e9
            res[name] = {"t": d.t, "planes_per_step": d.planes_per_step, "gcells": round(gc, 2),
                         "roofline_frac": round(gc / roof, 4)}
            del x, y
            torch.cuda.empty_cache()
        for name in ("bf16", "f16"):
            res[name]["speedup_vs_f32"] = round(res[name]["gcells"] / res["f32"]["gcells"], 3)
        f = gen.workload_grid(dim, *((small,) * dim))
        c = gen.coefficients(dim, r)
        w64 = oracle.sweep_f64(f.astype(np.float64), dim, r, c.astype(np.float64), iters)
        for name, dt, _ in dts:
            xs = torch.from_numpy(f).to(dt)
            got = s.run(xs.cuda(), iters).float().cpu().numpy().astype(np.float64)
            res[name]["accuracy"] = {"grid": [small] * dim, "iters": iters,
                                     "max_abs_vs_fp64": float(np.max(np.abs(got - w64))),
                                     "rel_l2_vs_fp64": float(np.linalg.norm(got - w64) / np.linalg.norm(w64))}
        out[key] = res
        s.close()
    assert st.stencil_get_device_status() == 0
    return out


def measure_batched(stream):
    """The 96-grid mixed batch (64 2D sides 512-8192, 32 3D sides 64-384, radius 1-4, FP32/BF16,
    100 iterations each; rows rounded down to 8 cells) as one stencil_run_batched call against
    the same grids swept one stencil_run after another."""
    import torch
    import paper_2002_05983_gb300 as st
    iters = 100
    items = gen.batch_list()
    stencils, bufs, batch = {}, [], []
    g = torch.Generator(device="cuda")
    g.manual_seed(100)
    for it in items:
        it["nx"] -= it["nx"] % 8
        key = (it["dim"], it["r"])
        if key not in stencils:
            stencils[key] = st.Stencil(it["dim"], it["r"], gen.coefficients(*key))
        shape = (it["ny"], it["nx"]) if it["dim"] == 2 else (it["nz"], it["ny"], it["nx"])
        dt = torch.bfloat16 if it["dtype"] == "bf16" else torch.float32
        x = torch.rand(shape, device="cuda", generator=g).to(dt)
        y = torch.empty_like(x)
        bufs.append((x, y))
        batch.append((stencils[key].handle, x.data_ptr(), y.data_ptr(), it["nx"], it["ny"], it["nz"], iters,
                      st.dtype_code(x)))
    sp = stream.cuda_stream
    cells = sum(b[3] * b[4] * b[5] for b in batch) * iters

    def singles():
        for h, xp, yp, nx, ny, nz, it_, code in batch:
            st.stencil_run(h, xp, yp, nx, ny, nz, it_, code, sp)

    t_single = _event_time(singles, 2, stream)
    ref = [y.clone() for _, y in bufs]
    t_batch = _event_time(lambda: st.stencil_run_batched(batch, sp), 3, stream)
    assert st.stencil_get_device_status() == 0
    same = sum(int(torch.equal(y, r)) for (_, y), r in zip(bufs, ref))
    res = {"grids": len(batch), "grids_2d": sum(1 for it in items if it["dim"] == 2), "iters": iters,
           "cell_updates": cells, "seconds_individual": round(t_single, 4), "seconds_batched": round(t_batch, 4),
           "gcells_individual": round(cells / t_single / 1e9, 1), "gcells_batched": round(cells / t_batch / 1e9, 1),
           "speedup_vs_individual": round(t_single / t_batch, 3),
           "grids_bit_identical_to_individual": f"{same}/{len(batch)}"}
    for s in stencils.values():
        s.close()
    return res


def model_accuracy_main(args):
    """Analytic model against measurement on the benchmark configurations (the paper's Table III
    "Model Accuracy" column, measured / estimated, and its model-guided choice of par_time,
    Section VI.A): per configuration and radius, measured / analytic time at the default
    schedule, the analytic model's best temporal degree against the measured best, and the
    regret of the analytic pick.  Every candidate is timed by stencil_tune's exhaustive mode
    (timing grids: the library's own, values do not change the speed)."""
    import torch
    import paper_2002_05983_gb300 as st
    from paper_2002_05983_gb300 import tune
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    confs = [("2D 16384^2 FP32", 2, 16384, st.STENCIL_F32, RADII), ("3D 512^3 FP32", 3, 512, st.STENCIL_F32, RADII),
             ("3D 768^3 BF16", 3, 768, st.STENCIL_BF16, (4,)), ("3D 768^3 FP16", 3, 768, st.STENCIL_F16, (4,)),
             ("2D 32768^2 BF16", 2, 32768, st.STENCIL_BF16, (4,)), ("2D 32768^2 FP16", 2, 32768, st.STENCIL_F16, (4,))]
    tdt = {st.STENCIL_F32: torch.float32, st.STENCIL_BF16: torch.bfloat16, st.STENCIL_F16: torch.float16}
    for name, dim, n, dt, radii in confs:
        shape = (n,) * dim
        nx, ny, nz = (n, n, 1) if dim == 2 else (n, n, n)
        x = torch.rand(shape, device="cuda").to(tdt[dt])
        out = torch.empty_like(x)
        for r in radii:
            s = st.Stencil(dim, r, gen.coefficients(dim, r))
            d = s.default_schedule(shape, dt)
            iters = 8 * d.t
            sec = _event_time(lambda: s.run(x, iters, out=out), 2, stream)
            meas_def = sec * 1e9 / (x.numel() * iters)
            ana_def = 2.0 ** float(st.stencil_schedule_features(s.handle, nx, ny, nz, dt, d)[11])
            _, rows = st.stencil_tune(s.handle, nx, ny, nz, dt, st.TUNE_EXHAUSTIVE, store=False, cap=512)
            meas = np.array([t.ns_per_cell for t in rows])
            ana = np.array([t.analytic_ns_per_cell for t in rows])
            per_t = {}
            for t, mv, av in zip(rows, meas, ana):
                k = int(t.sched.t)
                per_t.setdefault(k, [1e30, 1e30])
                per_t[k] = [min(per_t[k][0], mv), min(per_t[k][1], av)]
            best_meas_t = min(per_t, key=lambda k: per_t[k][0])
            best_ana_t = min(per_t, key=lambda k: per_t[k][1])
            ia, im = int(np.argmin(ana)), int(np.argmin(meas))
            _row(model_accuracy=True, config=name, dim=dim, r=r, default_t=d.t, default_planes_per_step=d.planes_per_step,
                 measured_over_analytic_at_default=round(meas_def / ana_def, 3),
                 gcells_default=round(1.0 / meas_def, 1), gcells_analytic_default=round(1.0 / ana_def, 1),
                 best_t_analytic=best_ana_t, best_t_measured=best_meas_t,
                 analytic_pick=dict(t=rows[ia].sched.t, planes_per_step=rows[ia].sched.planes_per_step,
                                    seg=rows[ia].sched.seg, rows_per_thread=rows[ia].sched.rows_per_thread),
                 measured_best=dict(t=rows[im].sched.t, planes_per_step=rows[im].sched.planes_per_step,
                                    seg=rows[im].sched.seg, rows_per_thread=rows[im].sched.rows_per_thread),
                 regret_analytic_pick=round(tune.regret_of(meas, ia), 4),
                 regret_default=round(max(meas_def / meas.min() - 1.0, 0.0), 4),
                 per_t={k: dict(measured_gcells=round(1.0 / v[0], 1), analytic_gcells=round(1.0 / v[1], 1))
                        for k, v in sorted(per_t.items())})
            s.close()
        del x, out
        torch.cuda.empty_cache()
    assert st.stencil_get_device_status() == 0
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the 3D, 16-bit storage and batch measurements that follow the headline")
    ap.add_argument("--suite", choices=["sweep2d", "sweep3d", "precision", "batch", "shared"], default=None,
                    help="other workloads: t sweeps, 16-bit storage, 96-grid batch, shared coefficients (JSON lines)")
    ap.add_argument("--radii", default="1,2,3,4",
                    help="radii of the sweep2d/sweep3d suites (1..6; the paper's range is 1..4)")
    ap.add_argument("--tune-eval", action="store_true",
                    help="measure all schedules of seeded problems, train the cost model, report regret")
    ap.add_argument("--model-accuracy", action="store_true",
                    help="analytic model vs measurement on the benchmark configurations (Table III form)")
    ap.add_argument("--case", default=None,
                    help="single sweep for profiling: dim:r:t:n:iters[:dtype[:rows_per_step]] (grid n^dim, t=0 auto)")
    args = ap.parse_args()
    if args.impl == "reference":
        return reference_main(args)
    if args.case:
        return case_main(args)
    if args.tune_eval:
        return tune_main(args)
    if args.model_accuracy:
        return model_accuracy_main(args)
    if args.suite:
        return suite_main(args)

    import torch
    import paper_2002_05983_gb300 as st
    from paper_2002_05983_gb300 import metrics

    world, rank, local = rank_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    # ---- inputs (seeded; 1 GiB, larger than L2 so no flush is needed between steps).  The
    # pinned host buffers are allocated and filled from CPUs next to this GPU, so that their
    # pages sit in the GPU's local host memory (reads from the far socket's memory measured
    # ~15 GB/s host-to-device against ~200 GB/s local).
    t0 = time.time()
    all_cpus = os.sched_getaffinity(0)
    near = gpu_local_cpus(local)
    if near:
        os.sched_setaffinity(0, near)
    host = torch.empty((NY, NX), dtype=torch.float32).pin_memory()
    gen.uniform_grid((NY, NX), out=host.numpy())
    host_out = torch.empty_like(host).pin_memory()
    host_out.zero_()
    if near:
        os.sched_setaffinity(0, all_cpus)
    x = host.cuda()
    out = torch.empty_like(x)
    log(f"rank {rank}: input ready in {time.time() - t0:.1f}s; pinned buffers allocated on "
        f"{len(near) if near else 'all'} CPUs next to GPU {local}")

    def copy_bandwidth(when):
        for name, (dst, src) in (("h2d", (x, host)), ("d2h", (host_out, out))):
            c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            c0.record()
            dst.copy_(src, non_blocking=True)
            c1.record()
            c1.synchronize()
            log(f"rank {rank}: {name} copy of {src.numel() * 4 / 2**30:.0f} GiB pinned {when}: "
                f"{src.numel() * 4 / c0.elapsed_time(c1) / 1e6:.1f} GB/s")

    copy_bandwidth("before the sweeps")
    pk = peaks()
    stencils = {r: st.Stencil(2, r, gen.coefficients(2, r)) for r in RADII}
    scheds = {r: stencils[r].default_schedule((NY, NX)) for r in RADII}
    stream = torch.cuda.current_stream()

    def step(ev=None):
        for r in RADII:
            if ev is not None:
                ev[r][0].record(stream)
            stencils[r].run(x, ITERS, out=out)
            if ev is not None:
                ev[r][1].record(stream)

    for _ in range(args.warmup):
        step()
    barrier()
    assert st.stencil_get_device_status() == 0

    evs = [{r: (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for r in RADII}
           for _ in range(args.steps)]
    e_start, e_stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    with Clocks(local) as clk:
        e_start.record(stream)
        for k in range(args.steps):
            step(evs[k])
        e_stop.record(stream)
        barrier()
    elapsed = e_start.elapsed_time(e_stop) / 1e3
    if st.stencil_get_device_status() != 0:
        raise RuntimeError("device status reports a timed-out kernel")
    elapsed = reduce_max(elapsed, dist, "cuda")

    per_r = {}
    for r in RADII:
        per_r[r] = sum(evs[k][r][0].elapsed_time(evs[k][r][1]) for k in range(args.steps)) / 1e3 / args.steps
    cells_step = NX * NY * ITERS * len(RADII)
    value = job_rate(cells_step * args.steps, world, elapsed) / 1e9
    flops_step = sum(NX * NY * ITERS * metrics.flop_per_cell(2, r) for r in RADII)

    # ---- end to end through the C ABI on pinned host buffers (copies inside the timed region)
    e2e_steps = max(1, args.steps // 2)
    copy_bandwidth("after the device-timed sweeps")
    for r in RADII:   # first calls per handle allocate its device and ping-pong buffers: keep them out
        stencils[r].run_host(host, host_out, 12)   # >= 2 passes at every degree used
    copy_bandwidth("after the end-to-end warm-up")
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        for r in RADII:
            stencils[r].run_host(host, host_out, ITERS)
    barrier()
    e2e_el = time.perf_counter() - t0
    e2e_el = reduce_max(e2e_el, dist, "cuda")
    copy_bandwidth("after the end-to-end runs")
    e2e = {"value": round(job_rate(cells_step * e2e_steps, world, e2e_el) / 1e9, 3), "unit": "GCell/s",
           "h2d_bytes_per_step": host.numel() * 4 * len(RADII),
           "d2h_bytes_per_step": host_out.numel() * 4 * len(RADII)}

    # ---- roofline of the dominant kernel (the radius with the longest time)
    rows = []
    launches = 0
    for r in RADII:
        t = scheds[r].t
        nl = -(-ITERS // t)
        launches += nl * args.steps
        sec = per_r[r]
        g = NX * NY * ITERS / sec / 1e9
        roof = metrics.roofline_cells(2, r, t, 4, pk["fp32_flops"], pk["hbm_gbs"] * 1e9) / 1e9
        rows.append({"r": r, "t": t, "planes_per_step": scheds[r].planes_per_step, "gcells": round(g, 2),
                     "gflops": round(g * metrics.flop_per_cell(2, r), 1),
                     "roofline_gcells": round(roof, 1), "roofline_frac": round(g / roof, 4),
                     "bound": metrics.roofline_bound(2, r, t, 4, pk["fp32_flops"], pk["hbm_gbs"] * 1e9),
                     "limiter": limiter_for(2, r, t, g * 8 / (t * pk["hbm_gbs"])),
                     "ms": round(sec * 1e3, 2)})
    dom = max(rows, key=lambda d: d["ms"])
    nl = -(-ITERS // dom["t"])
    launch_s = dom["ms"] / 1e3 / nl
    if dom["bound"] == "hbm":
        ach = NX * NY * 8 / launch_s / 1e9
        roofline = {"bound": "hbm", "achieved": round(ach, 1), "peak": pk["hbm_gbs"], "unit": "GB/s",
                    "peak_source": pk["hbm_src"] + " copy bandwidth (MEASURED_PEAKS.json hbm_gbs)"}
    else:
        ach = NX * NY * dom["t"] * metrics.flop_per_cell(2, dom["r"]) / launch_s / 1e12
        roofline = {"bound": "alu", "achieved": round(ach, 2), "peak": round(pk["fp32_flops"] / 1e12, 2),
                    "unit": "TFLOP/s", "peak_source": pk["fp32_src"]}
    roofline["frac"] = round(roofline["achieved"] / roofline["peak"], 4)
    roofline["kernel"] = f"sweep_kernel<2D, r={dom['r']}, t={dom['t']}, fp32>"
    roofline["traffic"] = traffic_for(2, dom["r"], dom["t"])
    roofline["algorithmic_bytes_per_launch"] = NX * NY * 8
    # `bound` names the lower roof of R(t); what limits the kernel in practice, from ncu's counters
    roofline["limiter"] = dom["limiter"]

    line = {"metric": METRIC, "value": round(value, 3), "unit": "GCell/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(elapsed / args.steps * 1e3, 2),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "grid": [NY, NX], "iters": ITERS, "radii": list(RADII),
                       "input": "uniform [0,1) from seed 0 (SplitMix64), coefficients seed 1",
                       "l2": "inputs larger than L2 (1 GiB grid), no flush",
                       "parallelism": f"replicas x{world}"},
            "gflops": round(flops_step * args.steps * world / elapsed / 1e9, 1),
            "per_radius": rows, "roofline": roofline, "e2e": e2e, "gpu_launches": launches,
            "peaks": {"fp32_tflops": round(pk["fp32_flops"] / 1e12, 2), "fp32_source": pk["fp32_src"],
                      "hbm_gbs": pk["hbm_gbs"], "hbm_source": pk["hbm_src"] + " (MEASURED_PEAKS.json)",
                      "copy_gbs_library_kernel": round(pk.get("copy_gbs_library", 0.0), 1)}}
    # ---- the other workloads (outside the timed region above): 3D, 16-bit storage, batch
    if not args.no_extra:
        t_extra = time.time()
        line["per_radius_3d"] = measure_3d(pk, stream)
        line["precision"] = measure_precision(pk, stream)
        line["batched"] = measure_batched(stream)
        log(f"rank {rank}: 3D, precision and batch measurements took {time.time() - t_extra:.1f}s")
    clk = clk.summary()
    if clk:
        line["clocks"] = clk
        if clk.get("power_w"):
            line["power"] = {"board_w_median": clk["power_w"],
                             "gflops_per_w": round(line["gflops"] / world / clk["power_w"], 2)}
    if rank == 0 and not args.no_cpu_baseline and world == 1:
        g, dt, cores, sample = oracle_leg(1, 0)
        line["cpu_baseline"] = {"value": round(g, 4), "unit": "GCell/s", "cores": cores, "kind": "oracle",
                                "sample": sample, "cpu": host_cpu()}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
