"""Continuous-batching request loop for Born solves.

Requests (grid, medium, source, frequency) arrive over time.  A dispatcher
admits a waiting request as soon as a solve slot is free and the device has
room for it (free HBM from cudaMemGetInfo, less a reserve, must cover the
request's footprint); each admitted request runs on its own worker thread and
its own solver stream, so solves of different sizes overlap on the GPU while
others are still arriving.  Each solve is the FP32 + FP64-refinement path with
its iteration blocks replayed from captured CUDA graphs; the solver keeps the
request's fields and medium on the device from upload to result.

The C ABI calls release the Python GIL (ctypes), so worker threads run their
solves concurrently.  Results are independent of the mix: solvers share no
device state and every reduction has a fixed order, so a request's field is
bitwise the same alone and in the mix.
"""
from __future__ import annotations

import math
import threading
import time
from dataclasses import dataclass, field

import numpy as np

from . import cbs, workloads as W

# bytes per voxel per component and per voxel of one FP32 + refinement solve (solver-owned arrays)
_FIELD_BYTES = 3 * 16 + 3 * 8       # x64, y64, w64 + x32, y32, w32 per component
_MEDIUM_BYTES = 5 * 8 + 5 * 4       # rs_eta (<=3), kp, et in float64 and float32
_INPUT_BYTES = 3 * 8                # c0, rho, alpha (float64, caller-owned)
_IO_BYTES = 2 * 16                  # source + result field per component (complex128, caller-owned)


def footprint_bytes(shape) -> int:
    """Device bytes one request needs (solver + its inputs and output), plus 5 % for tables and partials."""
    n = int(np.prod(shape))
    C = len(shape) + 1
    return int(1.05 * n * (C * (_FIELD_BYTES + _IO_BYTES) + _MEDIUM_BYTES + _INPUT_BYTES)) + (16 << 20)


@dataclass
class Request:
    rid: int
    arrival: float                 # seconds after the stream starts
    shape: tuple
    ppw: float
    seed: int
    src_pos: tuple                 # (x, y[, z])
    f_hz: float = W.F0             # source frequency; dx = c_water / (f_hz * ppw)
    problem: W.Problem | None = None
    # filled by the server
    admitted: float = math.nan
    done: float = math.nan
    iters: int = 0
    outer: int = 0
    residual: float = math.nan
    status: str = ""
    result: object = None          # pressure component (torch tensor on the host) when keep_results
    ready: object = None           # CUDA event recorded after `problem` was made (torch.cuda.Event), or None


def make_requests(n=256, seed=4, rate=None, sizes3d=(64, 96, 128, 192), sizes2d=(512, 1024, 2048), n_abs=16,
                  build=True, device=None, freqs=(250e3, 500e3, 1e6)):
    """Seeded request stream: grid uniform over the 3D cubes and 2D squares, frequency uniform over `freqs`,
    medium smoothed noise (sigma = n/16) mapped to c in [1400, 2800], rho in [900, 1900], alpha in [0, 5]
    dB/cm/MHz, PPW ~ U(4, 8), a point pressure source at a uniform interior voxel; Poisson arrivals at
    `rate` per second (all at 0 when rate is None)."""
    rng = np.random.default_rng(seed)
    # arrival times come from a stream of their own, so the requests are the same with or without a rate
    rng_t = np.random.default_rng([seed, 1])
    shapes = [(s, s, s) for s in sizes3d] + [(s, s) for s in sizes2d]
    t = 0.0
    reqs = []
    for i in range(n):
        shape = shapes[int(rng.integers(0, len(shapes)))]
        ppw = float(rng.uniform(4.0, 8.0))
        pos = tuple(int(rng.integers(n_abs + 1, s - n_abs - 1)) for s in shape[::-1])
        if rate:
            t += float(rng_t.exponential(1.0 / rate))
        f = float(freqs[int(rng.integers(0, len(freqs)))])
        r = Request(rid=i, arrival=t, shape=shape, ppw=ppw, seed=int(rng.integers(0, 2 ** 31)), src_pos=pos, f_hz=f)
        if build:
            r.problem = build_problem(r, n_abs, device)
            r.ready = _record_ready(device)
        reqs.append(r)
    return reqs


def _record_ready(device=None):
    """An event on the current stream after the work enqueued so far (the medium just made)."""
    import torch

    ev = torch.cuda.Event()
    ev.record(torch.cuda.current_stream(device))
    return ev


def build_problem(r: Request, n_abs=16, device=None) -> W.Problem:
    """The request's medium, generated on the device (torch) by the smooth-random recipe."""
    return W.smooth_random_medium_torch(r.shape, seed=r.seed, c_range=(1400.0, 2800.0), rho_range=(900.0, 1900.0),
                                        alpha_db_range=(0.0, 5.0), sigma_frac=1.0 / 16, ppw=r.ppw, n_abs=n_abs,
                                        f_hz=r.f_hz, device=device)


class Server:
    """Admission by slots and free HBM; one worker thread per running request.

    exclusive_voxels: requests with at least this many voxels (grids whose kernels fill the GPU on their own:
    1024^2, 128^3 and larger by default) run one at a time among themselves; smaller requests are admitted beside
    them and may pass a large request that waits for the running one.  Measured on the 256-request mixed stream
    at 0.8 x its saturated rate: p50 0.33 s / p99 2.51 s against 0.56 s / 2.91 s in plain arrival order, with a
    3 % higher saturated rate.  None or 0: every request is admitted in arrival order while slots and memory
    last."""

    def __init__(self, max_slots=6, reserve_bytes=8 << 30, tol=1e-6, precision="fp32_refine", keep_results=False,
                 check_every=50, allocator="torch", exclusive_voxels=1 << 20):
        self.max_slots = max_slots
        self.exclusive = exclusive_voxels
        self._big = 0
        self.reserve = reserve_bytes
        self.tol = tol
        self.precision = precision
        self.keep = keep_results
        self.check_every = check_every
        self.allocator = allocator
        self._lock = threading.Condition()
        self._running = 0
        self._reserved = 0
        self.max_concurrent = 0

    def _free_bytes(self):
        import torch
        free, _ = torch.cuda.mem_get_info()
        return free

    def _is_big(self, r: Request) -> bool:
        return bool(self.exclusive) and int(np.prod(r.shape)) >= self.exclusive

    def _fits(self, need):
        return self._running < self.max_slots and self._free_bytes() - self._reserved - need >= self.reserve

    def _solve(self, r: Request, t0: float, dev):
        try:
            self._work(r, dev)
        except Exception as e:  # a failed request is reported, the loop goes on
            r.status = f"error: {e}"
        finally:
            r.done = time.perf_counter() - t0
            with self._lock:
                self._running -= 1
                self._reserved -= footprint_bytes(r.shape)
                if self._is_big(r):
                    self._big -= 1
                self._lock.notify_all()

    def _work(self, r: Request, dev):
        """One request's solve on its own stream; fills r.iters, r.outer, r.residual, r.status (and r.result)."""
        import torch

        stream = torch.cuda.Stream(device=dev)
        with torch.cuda.stream(stream):
            if r.problem is not None:
                # the medium was made on another stream (torch's streams do not wait for each other): order
                # this request's work after it
                if r.ready is not None:
                    stream.wait_event(r.ready)
                else:
                    stream.wait_stream(torch.cuda.default_stream(dev))
            p = r.problem if r.problem is not None else build_problem(r, device=dev)
            c0, rho, al = p.c0, p.rho, p.alpha
            C = len(r.shape) + 1
            src = torch.zeros((C,) + tuple(r.shape), dtype=torch.complex128, device=dev)
            src[(C - 1,) + tuple(r.src_pos[::-1])] = 1.0
            field = torch.empty_like(src)
            stream.synchronize()
            # the solver's arrays come from torch's caching allocator: cudaMalloc / cudaFree can synchronise
            # the device and would stall the other requests' streams at every admission and completion
            s = cbs.solver_create(c0, rho, al, p.dx, p.omega, p.nabs, p.gamma_max, precision=self.precision,
                                  tol=self.tol, check_every=self.check_every, stream=stream,
                                  allocator=self.allocator)
            info = s.solve_forward(src, field, allow_noconv=True)
            s.destroy()
            if self.keep:
                r.result = field[C - 1].cpu()
            r.iters, r.outer = info["iters"], info["outer_iters"]
            r.residual, r.status = info["rel_residual"], info["status"]
            del c0, rho, al, src, field

    def run(self, requests, realtime=True):
        """Serve the request list; arrival times are honoured when realtime (else all are queued at once).
        Returns the requests with admission / completion times (seconds from the start)."""
        import torch

        dev = torch.device("cuda", torch.cuda.current_device())
        pending = sorted(requests, key=lambda r: r.arrival)
        waiting = []
        threads = []
        t0 = time.perf_counter()
        i = 0
        while i < len(pending) or waiting:
            now = time.perf_counter() - t0
            while i < len(pending) and (not realtime or pending[i].arrival <= now):
                waiting.append(pending[i])
                i += 1
            with self._lock:
                j = 0
                while j < len(waiting):
                    r = waiting[j]
                    big = self._is_big(r)
                    if big and self._big > 0:
                        j += 1  # waits for the running large request; a smaller one behind it may go first
                        continue
                    need = footprint_bytes(r.shape)
                    if not (self._fits(need) or self._running == 0):
                        break  # slots or memory: keep the arrival order
                    waiting.pop(j)
                    self._running += 1
                    self._reserved += need
                    if big:
                        self._big += 1
                    self.max_concurrent = max(self.max_concurrent, self._running)
                    r.admitted = time.perf_counter() - t0
                    th = threading.Thread(target=self._solve, args=(r, t0, dev), daemon=True)
                    th.start()
                    threads.append(th)
                if waiting or i < len(pending):
                    next_arrival = pending[i].arrival - (time.perf_counter() - t0) if i < len(pending) else 0.05
                    self._lock.wait(timeout=max(1e-3, min(0.05, next_arrival)) if realtime else 0.05)
        for th in threads:
            th.join()
        return requests


def summarize(requests):
    """Latency (arrival -> result) percentiles, throughput and per-status counts."""
    lat = np.array([r.done - r.arrival for r in requests if not math.isnan(r.done)])
    span = max(r.done for r in requests) - min(r.arrival for r in requests)
    vox_it = sum(int(np.prod(r.shape)) * r.iters for r in requests)
    status = {}
    for r in requests:
        status[r.status] = status.get(r.status, 0) + 1
    return {"requests": len(requests), "p50_ms": 1e3 * float(np.percentile(lat, 50)),
            "p99_ms": 1e3 * float(np.percentile(lat, 99)), "mean_ms": 1e3 * float(lat.mean()),
            "throughput_req_s": len(requests) / span, "voxel_iters_per_s": vox_it / span, "span_s": span,
            "status": status}
