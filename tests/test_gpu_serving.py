"""Continuous-batching request loop: requests of different grids, media and
frequencies admitted while others run give, per request, bitwise the same
field as when solved alone; latency and throughput are reported."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _stream(n=10, seed=12):
    from paper_2507_16087_gb300 import serving as S

    return S.make_requests(n=n, seed=seed, sizes3d=(64, 96), sizes2d=(256, 512), device="cuda:0")


def test_results_same_alone_and_in_the_mix():
    from paper_2507_16087_gb300 import serving as S

    alone = _stream()
    S.Server(max_slots=1, keep_results=True).run(alone, realtime=False)
    mixed = _stream()
    srv = S.Server(max_slots=6, keep_results=True)
    srv.run(mixed, realtime=False)
    assert srv.max_concurrent >= 2
    for a, b in zip(alone, mixed):
        assert a.status == b.status == "CBS_OK", (a.status, b.status)
        assert a.residual <= 1e-6 and a.iters == b.iters
        assert torch.equal(a.result, b.result), a.rid


def test_poisson_stream_reports_latency():
    from paper_2507_16087_gb300 import serving as S

    reqs = S.make_requests(n=12, seed=3, rate=20.0, sizes3d=(64,), sizes2d=(256, 512), device="cuda:0")
    S.Server(max_slots=4).run(reqs, realtime=True)
    summ = S.summarize(reqs)
    assert summ["status"] == {"CBS_OK": 12}
    assert 0 < summ["p50_ms"] <= summ["p99_ms"]
    for r in reqs:
        assert r.admitted >= r.arrival - 1e-3 and r.done > r.admitted


def test_footprint_admission_estimate_covers_solver_memory():
    from paper_2507_16087_gb300 import cbs, serving as S, workloads as W

    shape = (96, 96, 96)
    p = W.smooth_random_medium_torch(shape, seed=1, device="cuda:0")
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    s = cbs.solver_create(p.c0, p.rho, p.alpha, p.dx, p.omega, p.nabs, p.gamma_max, precision="fp32_refine")
    src = torch.zeros((4,) + shape, dtype=torch.complex128, device="cuda:0")
    field = torch.empty_like(src)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    used = free0 - free1
    assert used <= S.footprint_bytes(shape)
    s.destroy()
    del src, field


def test_freshly_made_media_are_ready_when_served():
    """A request's medium is made on the device just before it is served (another stream): the solve is ordered
    after it, so the largest grids' media are complete when the solver reads them."""
    from paper_2507_16087_gb300 import serving as S

    reqs = S.make_requests(n=4, seed=21, sizes3d=(192,), sizes2d=(2048,), device="cuda:0")
    S.Server(max_slots=4, exclusive_voxels=None).run(reqs, realtime=False)  # all four start at once
    assert [r.status for r in reqs] == ["CBS_OK"] * 4, [r.status for r in reqs]
