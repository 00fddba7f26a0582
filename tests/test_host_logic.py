"""Host-side logic that needs no GPU: the serving request stream and admission rule, the latency
summary, and the algorithmic byte counts the bench's roofline divides by."""
import math
import os
import sys

import numpy as np
import pytest

from paper_2507_16087_gb300 import serving as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_request_stream_is_seeded_and_well_formed():
    a = S.make_requests(n=64, seed=9, rate=5.0, build=False)
    b = S.make_requests(n=64, seed=9, rate=5.0, build=False)
    assert [(r.shape, r.ppw, r.seed, r.src_pos, r.arrival, r.f_hz) for r in a] == \
           [(r.shape, r.ppw, r.seed, r.src_pos, r.arrival, r.f_hz) for r in b]
    sizes = {(s, s, s) for s in (64, 96, 128, 192)} | {(s, s) for s in (512, 1024, 2048)}
    arrivals = [r.arrival for r in a]
    assert all(t1 > t0 for t0, t1 in zip(arrivals, arrivals[1:]))  # Poisson arrivals are strictly increasing
    assert {r.f_hz for r in a} == {250e3, 500e3, 1e6}
    for r in a:
        assert r.shape in sizes
        assert 4.0 <= r.ppw <= 8.0
        assert len(r.src_pos) == len(r.shape)
        # the source lies inside the absorbing layer's inner edge (n_abs = 16)
        assert all(16 < q < n - 17 for q, n in zip(r.src_pos, r.shape[::-1]))
    # mean inter-arrival time close to 1 / rate
    gaps = np.diff([0.0] + arrivals)
    assert abs(gaps.mean() - 0.2) < 0.08
    # all at time zero without a rate, and the same requests as with one (the saturation burst and the Poisson
    # stream of the serving bench are one request set)
    c = S.make_requests(n=64, seed=9, build=False)
    assert all(r.arrival == 0.0 for r in c)
    assert [(r.shape, r.ppw, r.seed, r.src_pos, r.f_hz) for r in a] == [(r.shape, r.ppw, r.seed, r.src_pos, r.f_hz) for r in c]


def test_footprint_grows_with_the_grid_and_covers_the_solver_arrays():
    f64 = S.footprint_bytes((64, 64, 64))
    f128 = S.footprint_bytes((128, 128, 128))
    assert f128 > 7.0 * f64  # 8x the voxels, plus a fixed 16 MiB for tables and partials
    n = 128 ** 3
    # x, y, w in float64 and float32 for 4 components, plus the caller's source and result
    assert f128 >= n * 4 * (3 * 16 + 3 * 8 + 2 * 16)
    assert S.footprint_bytes((1024, 1024)) > S.footprint_bytes((512, 512))


class _FakeServer(S.Server):
    def __init__(self, free, **kw):
        super().__init__(**kw)
        self.free = free

    def _free_bytes(self):
        return self.free


def test_admission_needs_a_slot_and_room_above_the_reserve():
    srv = _FakeServer(free=20 << 30, max_slots=2, reserve_bytes=8 << 30)
    assert srv._fits(4 << 30)
    assert not srv._fits(13 << 30)            # would dip into the reserve
    srv._reserved = 6 << 30                   # admitted requests that have not allocated yet
    assert not srv._fits(7 << 30)
    assert srv._fits(6 << 30)
    srv._running = 2                          # no free slot
    assert not srv._fits(1)


class _TimedServer(_FakeServer):
    """The admission loop with a fake worker: each request 'runs' for a time set by its size; the server
    records which requests ran at the same time."""

    def __init__(self, **kw):
        super().__init__(free=1 << 40, **kw)
        import threading
        self.guard = threading.Lock()
        self.live = set()
        self.overlaps = []      # (request, requests running when it started)
        self.order = []

    def _work(self, r, dev):
        import time
        with self.guard:
            self.overlaps.append((r.rid, set(self.live)))
            self.order.append(r.rid)
            self.live.add(r.rid)
        time.sleep(0.002 * (int(np.prod(r.shape)) >> 16))
        with self.guard:
            self.live.discard(r.rid)
        r.iters, r.status = 1, "CBS_OK"


def _mix(n=24):
    shapes = [(128, 128, 128), (16, 16, 16), (16, 16, 16), (192, 192, 192), (16, 16, 16), (1024, 1024)]
    return [S.Request(rid=i, arrival=0.0, shape=shapes[i % len(shapes)], ppw=6.0, seed=i, src_pos=(20, 20, 20))
            for i in range(n)]


def test_admission_in_arrival_order_without_the_exclusive_rule(monkeypatch):
    import torch
    monkeypatch.setattr(torch.cuda, "current_device", lambda: 0)
    reqs = _mix()
    srv = _TimedServer(max_slots=3, exclusive_voxels=None)
    srv.run(reqs, realtime=False)
    assert srv.order == [r.rid for r in reqs]                    # first come, first admitted
    assert all(r.status == "CBS_OK" for r in reqs)
    assert 2 <= srv.max_concurrent <= 3
    assert srv._running == 0 and srv._reserved == 0 and srv._big == 0


def test_large_requests_run_one_at_a_time_and_small_ones_pass_them(monkeypatch):
    import torch
    monkeypatch.setattr(torch.cuda, "current_device", lambda: 0)
    reqs = _mix()
    big = {r.rid for r in reqs if int(np.prod(r.shape)) >= 1 << 20}
    srv = _TimedServer(max_slots=3, exclusive_voxels=1 << 20)
    srv.run(reqs, realtime=False)
    assert all(r.status == "CBS_OK" for r in reqs) and sorted(srv.order) == [r.rid for r in reqs]
    for rid, running in srv.overlaps:
        if rid in big:
            assert not (running & big), (rid, running)           # never two large solves at once
    # small requests started while a large one ran, and some passed a waiting large one
    assert any(rid not in big and running & big for rid, running in srv.overlaps)
    assert srv.order != [r.rid for r in reqs]
    assert srv._running == 0 and srv._reserved == 0 and srv._big == 0


def test_summary_percentiles_and_throughput():
    reqs = []
    for i in range(10):
        r = S.Request(rid=i, arrival=float(i), shape=(64, 64, 64), ppw=6.0, seed=i, src_pos=(20, 20, 20))
        r.done = float(i) + 1.0 + 0.1 * i     # latencies 1.0 .. 1.9 s
        r.iters = 100
        r.status = "CBS_OK"
        reqs.append(r)
    out = S.summarize(reqs)
    assert out["requests"] == 10
    assert math.isclose(out["p50_ms"], 1450.0, rel_tol=1e-9)
    assert math.isclose(out["span_s"], 9.0 + 1.9)
    assert math.isclose(out["throughput_req_s"], 10 / 10.9)
    assert out["status"] == {"CBS_OK": 10}
    assert math.isclose(out["voxel_iters_per_s"], 10 * 64 ** 3 * 100 / 10.9)


def test_bench_algorithmic_bytes_per_voxel():
    sys.path.insert(0, ROOT)
    try:
        import bench
    finally:
        sys.path.remove(ROOT)
    b3 = bench.kernel_bytes_per_voxel(3, 4)
    # float32 3D, C = 4: a complex value is 8 bytes; medium = 3 rs + kp + et = 20 bytes
    assert b3["rows_fwd"] == 4 * 8 * 3 + 20 == 116
    assert b3["rows_inv"] == 116
    assert b3["axis_fwd"] == b3["axis_inv"] == b3["last_symbol"] == 64
    assert b3["plane_fwd"] == b3["plane_inv"] == 116
    it = sum(b3[k] for k in ("rows_fwd", "axis_fwd", "last_symbol", "axis_inv", "rows_inv"))
    assert it == 424
    b2 = bench.kernel_bytes_per_voxel(2, 4)
    assert b2["rows_fwd"] == 3 * 8 * 3 + 2 * 4 + 2 * 4  # 2 rs + kp + et


def _bench():
    sys.path.insert(0, ROOT)
    try:
        import bench
    finally:
        sys.path.remove(ROOT)
    return bench


def test_bench_model_bytes_and_fused_kernel_bytes():
    bench = _bench()
    m3 = bench.model_bytes_per_voxel(3, 4)
    # the survey's byte model: x, y, medium (c, rho, alpha) in and w out = 4*8*3 + 12
    assert m3["rows_fwd"] == m3["rows_inv"] == 108
    assert m3["axis_fwd"] == m3["last_symbol"] == m3["axis_inv"] == 64
    # fused update + next forward rows: w, x, y, medium in; x, w out
    assert m3["rows_inv_fwd"] == 4 * 8 * 5 + 12 == 172
    assert sum(m3[k] for k in ("axis_fwd", "last_symbol", "axis_inv", "rows_inv_fwd")) == 364
    assert bench.kernel_bytes_per_voxel(3, 4)["rows_inv_fwd"] == 180  # medium as stored: 3 rs + kp + et
    assert bench.model_bytes_per_voxel(3, 8)["rows_inv_fwd"] == 2 * 172  # float64 doubles every term


def test_profile_traffic_is_used_only_on_the_sources_it_was_taken_on(tmp_path):
    bench = _bench()
    h = bench.sources_hash()
    assert len(h) == 16 and h == bench.sources_hash()
    good = tmp_path / "good.md"
    good.write_text(f"text\ntraffic_bytes_per_launch sources={h}: rows_inv_fwd=301999360 last_symbol=68059392\n")
    d, stale = bench.profile_traffic(str(good))
    assert not stale and d == {"rows_inv_fwd": 301999360.0, "last_symbol": 68059392.0}
    other = tmp_path / "other.md"
    other.write_text("traffic_bytes_per_launch sources=0123456789abcdef: rows_inv_fwd=1\n")
    assert bench.profile_traffic(str(other)) == ({}, True)
    assert bench.profile_traffic(str(tmp_path / "missing.md")) == ({}, True)


@pytest.mark.parametrize("n", [64, 96])
def test_layered_inversion_workload_is_seeded_and_bounded(n):
    from paper_2507_16087_gb300 import workloads as W

    d1 = W.layered_inversion(n=n, n_abs=10)
    d2 = W.layered_inversion(n=n, n_abs=10)
    assert np.array_equal(d1["c0"], d2["c0"]) and np.array_equal(d1["rho"], d2["rho"])
    assert d1["c_layered"].min() >= 1400.0 and d1["c_layered"].max() <= 3000.0
    assert d1["rho_layered"].min() >= 900.0 and d1["rho_layered"].max() <= 2000.0
    # the perturbation is a few per cent of the layered model
    rel = np.abs(d1["c0"] / d1["c_layered"] - 1.0)
    assert rel.max() < 0.2 and rel.std() > 1e-3
