"""Benchmark of the split-preconditioned Born solver on one GB300.

Workload (one "step" = one full solve through every step of the hot path):
3D 128^3 grid, water (c 1500 m/s, rho 1000 kg/m^3) with a centred fluid sphere
of radius 24 cells (c 2200, rho 1600, 2 dB/cm/MHz), 500 kHz, 6 points per
wavelength, 20-cell absorbing layer, single-voxel pressure source 10 cells
inside the layer's inner edge; solved to a relative scaled residual of 1e-6.
A step is set-up (complex sound speed, staggered density, shifts, scaling),
the Born iterations, the float64 residual checks / refinement and the output
scaling, with the medium and source already resident on the device.

Metric: voxel-iterations per second (N_v * Born iterations / step time) of
the FP32 + FP64-refinement path; time to the 1e-6 residual for it and for the
plain FP64 path side by side.  --impl reference times the FP64 CPU oracle on
the host cores instead (bounded sample of the same workload).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "voxel-iters/s & time-to-1e-6 residual, FP32+refine vs FP64; p50/p99 latency"
UNIT = "voxel-iter/s"
WORKLOAD = "sphere3d_128: 128^3, sphere r=24 (c 2200, rho 1600, 2 dB/cm/MHz), point source, 20-cell layer, 6 PPW, tol 1e-6"
TOL = 1e-6


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.proc = None
        self.lines = []
        self.gpu = gpu_index

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    return ws, rank


def reduce_over_ranks(local_ms: float, local_units: float, device=None):
    """Replica aggregation: (max step time over ranks, total units over ranks).  With one process
    this is the identity; under torch.distributed (nccl on GPUs, gloo on CPU) it all-reduces."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(local_ms), float(local_units)
    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    u = torch.tensor([float(local_units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


# ------------------------------------------------------------------ oracle arm
def cpu_oracle_rate(problem, min_seconds=10.0, max_iter=200):
    """Voxel-iterations/s of the FP64 CPU oracle on the host cores, over a bounded sample: FP64 Born
    iterations of the same workload until at least min_seconds of CPU time (at most max_iter).
    Returns (rate, seconds, iterations, threads)."""
    from oracle import oracle as O

    P = O.Problem(problem.c0, problem.rho, problem.alpha, problem.dx, problem.omega, problem.nabs,
                  problem.gamma_max)
    y = P.scale_source(problem.source)
    n, dt = 0, 0.0
    while n == 0 or (dt < min_seconds and n < max_iter):
        k = 1 if n == 0 else max(1, min(max_iter - n, int(np.ceil((min_seconds - dt) / (dt / n)))))
        t0 = time.perf_counter()
        P.iterate(y, n_iter=k, nu=0.8)
        dt += time.perf_counter() - t0
        n += k
    return problem.n_voxels * n / dt, dt, n, O.max_threads()


def run_reference(args):
    ws, rank = _dist()
    if rank != 0:
        return 0
    from paper_2507_16087_gb300 import workloads as W

    p = W.sphere_128()
    rates = []
    for _ in range(args.warmup):
        cpu_oracle_rate(p, min_seconds=0.0)
    t_all, n_all = 0.0, 0
    for _ in range(args.steps):
        r, dt, n, cores = cpu_oracle_rate(p, min_seconds=5.0)
        rates.append(r)
        t_all += dt
        n_all += n
    value = float(p.n_voxels * n_all / t_all)
    sample = (f"{args.steps} steps of >= 5 s each: {n_all} FP64 Born iterations of the 128^3 sphere workload "
              f"(own FFT, OpenMP), {t_all:.1f} s")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * t_all / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD, "l2": "inputs larger than L2"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# -------------------------------------------------------------------- GPU arm
def sources_hash() -> str:
    """Hash of the CUDA sources (csrc/*.cu, *.cuh): a DRAM-traffic figure taken from a profile capture is
    reported only while the kernels are still the ones that capture measured."""
    import hashlib

    d = os.path.join(ROOT, "paper_2507_16087_gb300", "csrc")
    h = hashlib.sha256()
    off_path = {"measure.cu", "noalloc.cu"}  # not on the iteration's path
    for f in sorted(os.listdir(d)):
        if f.endswith((".cu", ".cuh")) and f not in off_path:
            h.update(f.encode())
            with open(os.path.join(d, f), "rb") as fh:
                h.update(fh.read())
    return h.hexdigest()[:16]


def profile_traffic(path=os.path.join(ROOT, "profiles", "born_iteration_sphere128.md")):
    """Per-launch DRAM read + write bytes of each iteration kernel from the committed ncu summary, which
    carries one line `traffic_bytes_per_launch sources=<hash>: kernel=bytes ...`.  Returns (dict, stale):
    the dict is empty and stale is True when the summary was taken on other kernel sources."""
    try:
        with open(path) as f:
            lines = [ln for ln in f if ln.startswith("traffic_bytes_per_launch")]
    except OSError:
        return {}, True
    if not lines:
        return {}, True
    head, _, body = lines[0].partition(":")
    src = head.split("sources=")[-1].strip()
    if src != sources_hash():
        return {}, True
    out = {}
    for tok in body.split():
        k, _, v = tok.partition("=")
        try:
            out[k] = float(v)
        except ValueError:
            pass
    return out, False


def kernel_bytes_per_voxel(D=3, fp=4):
    """Bytes per voxel each kernel of one iteration reads and writes as built (fields and the per-voxel
    medium arrays it streams: rs_eta per velocity component, kp and et for pressure)."""
    C = D + 1
    cb = 2 * fp               # one complex value
    medium = D * fp + 2 * fp  # rs_eta per velocity component + (kp, et) for pressure
    return {"rows_fwd": C * cb * 3 + medium,   # x, y in; w out
            "axis_fwd": C * cb * 2, "last_symbol": C * cb * 2, "axis_inv": C * cb * 2,
            "rows_inv": C * cb * 3 + medium,   # w, x in; x out
            "plane_fwd": C * cb * 3 + medium,  # x-y plane kernels: the same reads and writes as the row kernels
            "plane_inv": C * cb * 3 + medium,
            "rows_inv_fwd": C * cb * 5 + medium}  # w, x, y in; x, w out (update + next forward transform)


def model_bytes_per_voxel(D=3, fp=4):
    """The byte model of the method's passes: a kernel that reads x, y and the medium (c, rho, alpha in the
    working precision) and writes w moves C*3 complex values + 3 reals per voxel (108 B in float32 3D);
    a transform-only pass reads and writes w (64 B); the fused update + next forward row pass reads w, x, y
    and the medium and writes x and w (172 B)."""
    C = D + 1
    cb = 2 * fp
    medium = 3 * fp
    return {"rows_fwd": C * cb * 3 + medium, "axis_fwd": C * cb * 2, "last_symbol": C * cb * 2,
            "axis_inv": C * cb * 2, "rows_inv": C * cb * 3 + medium, "plane_fwd": C * cb * 3 + medium,
            "plane_inv": C * cb * 3 + medium, "rows_inv_fwd": C * cb * 5 + medium}


def run_gpu(args):
    import torch

    from paper_2507_16087_gb300 import cbs, workloads as W

    ws, rank = _dist()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group("nccl")
    dev = torch.device("cuda", torch.cuda.current_device())
    p = W.sphere_128()
    Nv = p.n_voxels
    T = lambda a, dt=torch.float64: torch.tensor(np.ascontiguousarray(a), dtype=dt, device=dev)  # noqa: E731
    c0, rho, al = T(p.c0), T(p.rho), T(p.alpha)
    src = T(p.source, torch.complex128)
    field = torch.zeros((4,) + p.shape, dtype=torch.complex128, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    kw = dict(tol=TOL, check_every=args.check_every, tol_inner=args.tol_inner, nu=args.nu)

    def solve(precision):
        s = cbs.solver_create(c0, rho, al, p.dx, p.omega, p.nabs, p.gamma_max, precision=precision, **kw)
        info = s.solve_forward(src, field)
        s.destroy()
        return info

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()

    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        solve("fp32_refine")
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    times, iters, launches, infos = [], [], 0, []
    for _ in range(args.steps):
        flush.zero_()
        barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        info = solve("fp32_refine")
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        times.append(e0.elapsed_time(e1))
        iters.append(info["iters"])
        launches += info["kernel_launches"]
        infos.append(info)
    clk = clocks.stop()
    t_ms = np.array(times)
    step_ms, units = reduce_over_ranks(float(t_ms.mean()), Nv * float(np.mean(iters)), device=dev)
    value = units / (step_ms / 1e3)

    # plain FP64 side by side (one warm-up, one timed)
    fp64 = None
    if not args.no_fp64:
        solve("fp64")
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        i64 = solve("fp64")
        e1.record(stream)
        torch.cuda.synchronize()
        t64 = e0.elapsed_time(e1)
        # the float64 path is bound by the FP64 pipes: its flop rate (5 log2(N_v) flops per point per transform,
        # forward and inverse, C components, plus ~100 for the symbol and the pointwise steps) against the
        # measured FP64 FMA rate of this GPU
        fp64_peak = cbs.fp64_rate()
        flops_per_vi = 2 * 4 * 5 * np.log2(Nv) + 100
        fp64_tflops = flops_per_vi * Nv * i64["iters"] / (t64 / 1e3) / 1e12
        fp64 = {"time_to_1e-6_ms": t64, "iters": i64["iters"], "rel_residual": i64["rel_residual"],
                "voxel_iters_per_s": Nv * i64["iters"] / (t64 / 1e3),
                "roofline": {"bound": "fp64", "achieved": fp64_tflops, "peak": fp64_peak, "unit": "TFLOP/s",
                             "frac": fp64_tflops / fp64_peak, "peak_kind": "measured FP64 FMA chains (cbs_fp64_rate)",
                             "flops_per_voxel_iter": flops_per_vi}}

    # per-kernel times (CUDA events on the solver's stream) for the roofline
    s = cbs.solver_create(c0, rho, al, p.dx, p.omega, p.nabs, p.gamma_max, precision="fp32_refine", **kw)
    y = torch.zeros_like(field)
    s.scale_source(src, y)
    x = torch.zeros_like(field)
    kt = s.time_kernels(y, x, 5)
    kt = s.time_kernels(y, x, 20)
    s.destroy()
    # the cuFFT comparison build of the same iteration (timed only), beside the fused iteration replayed from
    # its captured graphs as a solve runs it
    s = cbs.solver_create(c0, rho, al, p.dx, p.omega, p.nabs, p.gamma_max, precision="fp32_refine", **kw)
    x.zero_()
    s.cufft_iterate(y, x, 3)
    cufft_ms = s.cufft_iterate(y, x, 20)
    x.zero_()
    s.born_iterate(y, x, 50)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    s.born_iterate(y, x, 200)
    e1.record(stream)
    torch.cuda.synchronize()
    own_ms = e0.elapsed_time(e1) / 200
    s.destroy()
    cufft = {"iteration_ms": cufft_ms, "voxel_iters_per_s": Nv / (cufft_ms / 1e3), "own_iteration_ms": own_ms,
             "own_voxel_iters_per_s": Nv / (own_ms / 1e3), "speedup_vs_cufft": cufft_ms / own_ms,
             "what": "same float32 iteration: cuFFT batched C2C plans + plain pointwise kernels (stream launches)"}
    bpv = model_bytes_per_voxel(3, 4)
    kbpv = kernel_bytes_per_voxel(3, 4)
    peak, peak_kind = _peaks()
    top = max((k for k in kt if bpv.get(k, 0) > 0), key=lambda k: kt[k])
    achieved = bpv[top] * Nv / (kt[top] / 1e3) / 1e9
    achieved_k = kbpv[top] * Nv / (kt[top] / 1e3) / 1e9
    iter_ms = sum(kt.values())
    traffic, stale = profile_traffic()
    per_kernel = {k: {"ms": kt[k], "model_GBs": bpv[k] * Nv / (kt[k] / 1e3) / 1e9,
                      "frac": bpv[k] * Nv / (kt[k] / 1e3) / 1e9 / peak} for k in kt if bpv.get(k, 0) > 0}
    roof = {"bound": "hbm", "kernel": top, "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "peak_kind": peak_kind, "traffic": traffic.get(top),
            "traffic_source": "profiles/born_iteration_sphere128.md" if not stale else
                              "null: the committed capture was taken on other kernel sources",
            "sources": sources_hash(),
            "algorithmic_bytes": bpv[top] * Nv, "bytes_per_voxel": bpv[top],
            "kernel_bytes_per_voxel": kbpv[top], "achieved_kernel_bytes": achieved_k,
            "frac_kernel_bytes": achieved_k / peak, "kernel_ms": kt, "per_kernel": per_kernel,
            "iteration_ms": iter_ms,
            "iteration_frac": sum(bpv[k] for k in kt) * Nv / (iter_ms / 1e3) / 1e9 / peak,
            "iteration_frac_compulsory": 108 * Nv / (iter_ms / 1e3) / 1e9 / peak}

    # the largest configuration's grid (512^3, float32 iterations): per-kernel event times of a few iterations
    # on a sphere-inclusion medium (an iteration's time does not depend on the medium), against the same byte model
    large = None
    if not args.no_large and rank == 0:
        n = 512
        pl = W.inclusion_medium((n, n, n), 120, 1800.0, 1300.0, 1.0, ppw=6.0, n_abs=24)
        sl = cbs.solver_create(T(pl.c0), T(pl.rho), T(pl.alpha), pl.dx, pl.omega, pl.nabs, pl.gamma_max,
                               precision="fp32_refine", **kw)
        del pl
        yl = torch.zeros((4, n, n, n), dtype=torch.complex128, device=dev)
        yl[3, n // 2, n // 2, 30] = 1.0
        xl = torch.zeros_like(yl)
        sl.time_kernels(yl, xl, 1)
        ktl = sl.time_kernels(yl, xl, 3)
        sl.destroy()
        del yl, xl
        torch.cuda.empty_cache()
        it_ms = sum(ktl.values())
        nl = float(n) ** 3
        top_l = max(ktl, key=lambda k: ktl[k])
        large = {"shape": [n, n, n], "kernel_ms": ktl, "iteration_ms": it_ms,
                 "voxel_iters_per_s": nl / (it_ms / 1e3),
                 "iteration_frac": sum(bpv[k] for k in ktl) * nl / (it_ms / 1e3) / 1e9 / peak,
                 "per_kernel_frac": {k: bpv[k] * nl / (ktl[k] / 1e3) / 1e9 / peak for k in ktl},
                 "top_kernel": top_l}

    # end to end through the public API with host buffers (pinned), copies inside the timed region
    hc = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in (p.c0, p.rho, p.alpha)]
    hs = torch.from_numpy(np.ascontiguousarray(p.source)).pin_memory()
    hout = torch.empty((4,) + p.shape, dtype=torch.complex128).pin_memory()
    e2e_t = []
    side = torch.cuda.Stream(device=dev)
    for k in range(3):  # the last one is timed in the steady state: its device tensors reuse freed cached blocks
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        cur = torch.cuda.current_stream()
        dc = [a.to(dev, non_blocking=True) for a in hc]
        # the source is needed only by the solve: its copy runs on a side stream while the solver is made
        # (set-up reads only the medium)
        with torch.cuda.stream(side):
            ds = hs.to(dev, non_blocking=True)
        fld = torch.empty((4,) + p.shape, dtype=torch.complex128, device=dev)
        s = cbs.solver_create(dc[0], dc[1], dc[2], p.dx, p.omega, p.nabs, p.gamma_max, precision="fp32_refine", **kw)
        cur.wait_stream(side)
        ds.record_stream(cur)
        ie = s.solve_forward(ds, fld)
        hout.copy_(fld, non_blocking=True)
        torch.cuda.synchronize()
        s.destroy()
        e2e_t.append(time.perf_counter() - t0)
        del dc, ds, fld, s
    h2d = sum(a.numel() * a.element_size() for a in hc) + hs.numel() * hs.element_size()
    d2h = hout.numel() * hout.element_size()
    e2e = {"value": Nv * ie["iters"] / e2e_t[-1], "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
           "time_to_1e-6_ms": 1e3 * e2e_t[-1]}

    serving = None
    if args.serve_sample > 0:
        serving = serving_measure(args.serve_sample, seed=4, max_slots=args.slots,
                                  exclusive_voxels=args.serve_exclusive)

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        from oracle import oracle as O

        rate, dt, n_cpu, cores = cpu_oracle_rate(p, min_seconds=10.0)
        O.set_threads(1)
        rate1, dt1, n1, _ = cpu_oracle_rate(p, min_seconds=5.0)
        O.set_threads(cores)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{n_cpu} FP64 Born iterations of the same 128^3 workload ({dt:.1f} s)",
               "single_thread": {"value": rate1, "unit": UNIT, "cores": 1,
                                 "sample": f"{n1} FP64 Born iterations, one thread ({dt1:.1f} s)"}}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "c64 inner / f64 refine", "data": "synthetic",
                "config": {"workload": WORKLOAD, "precision": "fp32_refine", "l2": "flushed (256 MB write) between steps",
                           "parallelism": "replicas" if ws > 1 else "single"},
                "time_to_1e-6_ms": step_ms, "iters": float(np.mean(iters)),
                "outer_iters": infos[-1]["outer_iters"], "rel_residual": infos[-1]["rel_residual"],
                "setup_ms": infos[-1]["t_setup_ms"], "fp64": fp64, "roofline": roof, "cpu_baseline": cpu,
                "e2e": e2e, "gpu_launches": launches, "clocks": clk, "serving": serving, "cufft_baseline": cufft,
                "large_grid": large}
        print(json.dumps(line))
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def run_kernels(args):
    """Per-kernel device times of FP32 Born iterations on the bench workload (a short command for
    profilers); prints one JSON line."""
    import torch

    from paper_2507_16087_gb300 import cbs, workloads as W

    dev = torch.device("cuda", 0)
    if args.shape:
        shape = tuple(int(v) for v in args.shape.split(","))
        p = W.smooth_random_medium(shape, seed=1, n_abs=16)
        p.source = W.point_source(shape, tuple(s // 3 for s in shape[::-1]))
    else:
        p = W.sphere_128()
    T = lambda a, dt=torch.float64: torch.tensor(np.ascontiguousarray(a), dtype=dt, device=dev)  # noqa: E731
    prec = "fp64" if args.precision == "fp64" else "fp32_refine"
    s = cbs.solver_create(T(p.c0), T(p.rho), T(p.alpha), p.dx, p.omega, p.nabs, p.gamma_max, precision=prec, tol=TOL)
    src = T(p.source, torch.complex128)
    y = torch.zeros((p.ndim + 1,) + p.shape, dtype=torch.complex128, device=dev)
    s.scale_source(src, y)
    x = torch.zeros_like(y)
    kt = s.time_kernels(y, x, args.iters)
    s.destroy()
    print(json.dumps({"mode": "kernels", "shape": list(p.shape), "precision": prec, "iters": args.iters,
                      "kernel_ms": kt, "iteration_ms": sum(kt.values())}))
    return 0


def serving_measure(n_requests, seed=4, n_sat=None, max_slots=6, exclusive_voxels=1 << 20):
    """Serving stream: the saturated throughput from the first n_sat requests of the same stream (all queued at
    once; the whole stream by default), then the n_requests as Poisson arrivals at 0.8 x that rate; p50 / p99
    latency over all of them and the aggregate throughput.  Beside it, each grid size solved alone (one request
    per size, nothing else on the GPU) gives the throughput a one-request-at-a-time server would reach on the
    same stream; the saturated burst's own voxel-iteration rate is the concurrent server's capacity to set
    beside it (the Poisson stream's aggregate is bounded by the offered load).  exclusive_voxels: the server runs
    requests of at least that many voxels one at a time among themselves (None or 0: arrival order only)."""
    import torch

    from paper_2507_16087_gb300 import serving as S

    dev = torch.device("cuda", torch.cuda.current_device())
    burst = S.make_requests(n=n_sat or n_requests, seed=seed, device=dev)
    S.Server(max_slots=max_slots, exclusive_voxels=exclusive_voxels).run(burst, realtime=False)
    sat = S.summarize(burst)
    rate = 0.8 * sat["throughput_req_s"]
    reqs = S.make_requests(n=n_requests, seed=seed, rate=rate, device=dev)
    srv = S.Server(max_slots=max_slots, exclusive_voxels=exclusive_voxels)
    srv.run(reqs, realtime=True)
    out = S.summarize(reqs)
    # one request of each grid size alone (the first of that size in the stream, same medium and source):
    # seconds per voxel-iteration of that size with nothing else on the GPU
    alone, alone_status = {}, {}
    for r in reqs:
        if r.shape in alone_status:
            continue
        one = S.Request(rid=-1, arrival=0.0, shape=r.shape, ppw=r.ppw, seed=r.seed, src_pos=r.src_pos, f_hz=r.f_hz)
        one.problem = S.build_problem(one, device=dev)
        torch.cuda.synchronize()
        S.Server(max_slots=1).run([one], realtime=False)
        alone_status["x".join(map(str, r.shape))] = one.status
        if one.status == "CBS_OK" and one.iters > 0:
            alone[r.shape] = (one.done - one.admitted) / (int(np.prod(r.shape)) * one.iters)
    ok = [r for r in reqs if r.shape in alone]
    serial_s = sum(alone[r.shape] * int(np.prod(r.shape)) * r.iters for r in ok)
    vox_it = sum(int(np.prod(r.shape)) * r.iters for r in ok)
    out.update({"arrival_rate_req_s": rate, "saturated_req_s": sat["throughput_req_s"], "saturation_burst": n_sat,
                "saturated_voxel_iters_per_s": sat["voxel_iters_per_s"],
                "max_concurrent": srv.max_concurrent, "max_slots": max_slots, "exclusive_voxels": exclusive_voxels,
                "one_at_a_time_voxel_iters_per_s": vox_it / serial_s if serial_s > 0 else None,
                "alone_voxel_iters_per_s": {"x".join(map(str, k)): 1.0 / v for k, v in alone.items()},
                "alone_status": alone_status,
                "grids": "64^3/96^3/128^3/192^3, 512^2/1024^2/2048^2; 250 kHz/500 kHz/1 MHz; FP32+refine to 1e-6"})
    return out


def run_serve(args):
    out = serving_measure(args.requests, seed=4, n_sat=args.sat_requests or None, max_slots=args.slots,
                          exclusive_voxels=args.serve_exclusive)
    out["mode"] = "serve"
    print(json.dumps(out))
    return 0


def run_sweep(args):
    """Convergence versus contrast (a central disc in c or in rho, line source): FP32 + refinement
    iterations to a 1e-6 residual for each contrast; one JSON line."""
    import torch

    from paper_2507_16087_gb300 import cbs, workloads as W

    dev = torch.device("cuda", 0)
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)  # noqa: E731
    rows = []
    cases = [("c", d) for d in (0.0, 250.0, 500.0, 1000.0, 2000.0)] + [("rho", d) for d in (500.0, 1000.0, 2000.0, 4000.0)]
    for kind, d in cases:
        p = W.disc_perturbation(n=256, dc=d if kind == "c" else 0.0, drho=d if kind == "rho" else 0.0)
        for rule in (cbs.CBS_SHIFT_MIDRANGE, cbs.CBS_SHIFT_MEC):
            s = cbs.solver_create(T(p.c0), T(p.rho), T(p.alpha), p.dx, p.omega, p.nabs, p.gamma_max,
                                  precision="fp32_refine", tol=TOL, shift_rule=rule, max_iter=200000)
            field = torch.zeros((3,) + p.shape, dtype=torch.complex128, device=dev)
            info = s.solve_forward(T(p.source), field, allow_noconv=True)
            s.destroy()
            rows.append({"kind": kind, "delta": d, "shift": "mec" if rule else "midrange", "iters": info["iters"],
                         "rel_residual": info["rel_residual"], "ms": info["t_solve_ms"]})
    e1 = W.three_discs()
    s = cbs.solver_create(T(e1.c0), T(e1.rho), T(e1.alpha), e1.dx, e1.omega, e1.nabs, e1.gamma_max,
                          precision="fp32_refine", tol=TOL, max_iter=400000)
    field = torch.zeros((3,) + e1.shape, dtype=torch.complex128, device=dev)
    i1 = s.solve_forward(T(e1.source), field, allow_noconv=True)
    s.destroy()
    print(json.dumps({"mode": "sweep", "grid": "256^2, 6 PPW, 16-cell layer, disc r=32, line source", "rows": rows,
                      "three_discs": {"iters": i1["iters"], "rel_residual": i1["rel_residual"],
                                      "ms": i1["t_solve_ms"], "status": i1["status"]}}))
    return 0


def run_cpu(args):
    """FP64 CPU oracle voxel-iterations/s at every configuration size, all host cores and one thread:
    Born iterations of a seeded medium until a few seconds of work (at most 20 iterations); 512^3 all
    cores only when the host has the memory for it (one iteration takes tens of seconds there, one
    thread several minutes).  Prints one JSON line."""
    from oracle import oracle as O
    from paper_2507_16087_gb300 import workloads as W

    def mem_gb():
        try:
            with open("/proc/meminfo") as f:
                for ln in f:
                    if ln.startswith("MemAvailable:"):
                        return int(ln.split()[1]) / 2 ** 20
        except OSError:
            pass
        return 0.0

    cores = O.max_threads()
    sizes = [(128, 128), (512, 512), (1024, 1024), (2048, 2048), (64,) * 3, (96,) * 3, (128,) * 3, (192,) * 3]
    if args.n >= 512 and mem_gb() > 80:
        sizes.append((512,) * 3)
    rows = []
    for shape in sizes:
        nv = int(np.prod(shape))
        if len(shape) == 3 and shape[0] >= 512:
            p = W.inclusion_medium(shape, shape[0] // 4, 1800.0, 1300.0, 1.0, n_abs=24)
        else:
            p = W.smooth_random_medium(shape, seed=9, n_abs=16)
        src = np.zeros((len(shape) + 1,) + shape, dtype=np.complex128)
        src[(len(shape),) + tuple(s // 3 for s in shape)] = 1.0
        p.source = src
        row = {"shape": list(shape), "voxels": nv}
        for threads, key, secs in ((cores, "all_cores", 3.0), (1, "one_thread", 3.0)):
            if threads == 1 and nv > 2 ** 25:
                row[key] = None
                continue
            O.set_threads(threads)
            rate, dt, n, used = cpu_oracle_rate(p, min_seconds=secs, max_iter=20)
            row[key] = {"voxel_iters_per_s": rate, "iters": n, "seconds": dt, "threads": used}
        O.set_threads(cores)
        rows.append(row)
        print(json.dumps(row), file=sys.stderr, flush=True)
    print(json.dumps({"mode": "cpu", "cores": cores, "rows": rows}))
    return 0


def run_skull(args):
    """512^3 transcranial-like workload (shell + bowl, 24-cell layer): one FP32 + FP64-refinement solve to
    a 1e-6 residual; prints one JSON line with iterations, time, voxel-iter/s, the float64 residual
    recomputed through residual_norm, and per-kernel times."""
    import torch

    from paper_2507_16087_gb300 import cbs, workloads as W

    t0 = time.perf_counter()
    p = W.skull_shell(n=args.n)
    t_gen = time.perf_counter() - t0
    dev = torch.device("cuda", 0)
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)  # noqa: E731
    c0, rho, al = T(p.c0), T(p.rho), T(p.alpha)
    src = T(p.source)
    del p.source
    field = torch.zeros_like(src)
    s = cbs.solver_create(c0, rho, al, p.dx, p.omega, p.nabs, p.gamma_max, precision="fp32_refine", tol=TOL,
                          nu=args.nu, check_every=args.check_every)
    info = s.solve_forward(src, field)
    res = s.residual_norm(field, src)
    y = torch.zeros_like(src)
    s.scale_source(src, y)
    x = torch.zeros_like(src)
    kt = s.time_kernels(y, x, 3)
    s.destroy()
    Nv = int(np.prod(p.shape))
    print(json.dumps({"mode": "skull", "n": args.n, "voxels": Nv, "iters": info["iters"],
                      "outer_iters": info["outer_iters"], "rel_residual": info["rel_residual"],
                      "residual_recomputed": res, "time_to_1e-6_ms": info["t_solve_ms"],
                      "setup_ms": info["t_setup_ms"], "voxel_iters_per_s": Nv * info["iters"] / (info["t_solve_ms"] / 1e3),
                      "kernel_ms": kt, "bowl_voxels": p.meta["bowl_voxels"], "generate_s": t_gen,
                      "device_mem_gb": torch.cuda.max_memory_allocated() / 1e9}))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--check-every", type=int, default=50)
    ap.add_argument("--tol-inner", type=float, default=1e-4)
    ap.add_argument("--nu", type=float, default=0.8)
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-large", action="store_true", help="skip the 512^3 per-kernel timing leg")
    ap.add_argument("--mode", default="bench", choices=["bench", "kernels", "skull", "serve", "sweep", "cpu"])
    ap.add_argument("--requests", type=int, default=256)
    ap.add_argument("--sat-requests", type=int, default=0, help="requests of the saturation burst (0: the whole stream)")
    ap.add_argument("--slots", type=int, default=6)
    ap.add_argument("--serve-exclusive", type=int, default=1 << 20,
                    help="serving: requests of at least this many voxels run one at a time among themselves (0: off)")
    ap.add_argument("--serve-sample", type=int, default=256)
    ap.add_argument("--n", type=int, default=512)
    ap.add_argument("--iters", type=int, default=3)
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--shape", default="", help="kernels mode: numpy grid shape, e.g. 2048,2048 (default: the 128^3 sphere)")
    args = ap.parse_args()
    if args.mode == "kernels":
        return run_kernels(args)
    if args.mode == "skull":
        return run_skull(args)
    if args.mode == "serve":
        return run_serve(args)
    if args.mode == "sweep":
        return run_sweep(args)
    if args.mode == "cpu":
        return run_cpu(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
