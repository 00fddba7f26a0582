"""GPU adjoint / gradient path: the medium_gradient kernel against the oracle's
formula, torch.autograd through solve_forward / solve_adjoint against the
oracle gradient, and central finite differences (relative step 1e-4) of the
misfit on the layered-inversion workload (5 slabs + 3 % smoothed perturbation,
8 sources, 64 receivers)."""
import numpy as np
import pytest

from oracle import gradient as OG
from oracle import oracle as O
from paper_2507_16087_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def T(a):
    a = np.ascontiguousarray(a)
    return torch.tensor(a, device=DEV)


@pytest.mark.parametrize("shape", [(24, 32), (12, 16, 24)])
def test_medium_gradient_kernel_matches_oracle_formula(shape):
    from paper_2507_16087_gb300 import cbs

    p = W.smooth_random_medium(shape, seed=41, n_abs=3)
    s = cbs.solver_create(T(p.c0), T(p.rho), T(p.alpha), p.dx, p.omega, p.nabs, p.gamma_max)
    src = W.random_source(shape, 42)[None]
    X = W.random_source(shape, 43)[None]
    L = W.random_source(shape, 44)[None]
    gc = torch.zeros(shape, dtype=torch.float64, device=DEV)
    gr = torch.zeros_like(gc)
    s.medium_gradient(T(p.c0), T(p.rho), T(p.alpha), T(src[0]), T(X[0]), T(L[0]), gc, gr)
    rc, rr = OG.medium_gradient(p.c0, p.rho, p.alpha, p.omega, p.nabs, p.gamma_max, src, X, L)
    assert np.linalg.norm(gc.cpu().numpy() - rc) <= 1e-12 * np.linalg.norm(rc)
    assert np.linalg.norm(gr.cpu().numpy() - rr) <= 1e-12 * np.linalg.norm(rr)
    # accumulate adds
    s.medium_gradient(T(p.c0), T(p.rho), T(p.alpha), T(src[0]), T(X[0]), T(L[0]), gc, gr, accumulate=True)
    assert np.linalg.norm(gc.cpu().numpy() - 2 * rc) <= 1e-12 * np.linalg.norm(rc)


def _problem(n, n_abs, src_grid=(4, 2)):
    d = W.layered_inversion(n=n, n_abs=n_abs, src_grid=src_grid, rec_grid=(8, 8))
    return d


def _data(d, precision, tol):
    from paper_2507_16087_gb300 import autograd as AG

    with torch.no_grad():
        f = AG.helmholtz_fields(T(d["c_layered"]), T(d["rho_layered"]), T(d["alpha"]), T(d["sources"]), d["dx"],
                                d["omega"], d["nabs"], d["gamma_max"], precision=precision, tol=tol)
    rec = tuple(torch.tensor(r, device=DEV) for r in d["receivers"])
    return f[:, -1][(slice(None),) + rec].clone(), rec


def test_autograd_gradient_matches_oracle_small():
    from paper_2507_16087_gb300 import autograd as AG

    d = _problem(24, 4, src_grid=(2, 1))
    d["gamma_max"] = 0.5 * d["omega"]  # a 4-cell layer at full strength converges slowly; the check needs none
    rng = np.random.default_rng(24)
    nr = d["receivers"][0].size
    data_h = 1e-3 * (rng.standard_normal((2, nr)) + 1j * rng.standard_normal((2, nr)))
    data = T(data_h)
    rec = tuple(torch.tensor(r, device=DEV) for r in d["receivers"])
    c0 = T(d["c0"]).requires_grad_(True)
    rho = T(d["rho"]).requires_grad_(True)
    f = AG.helmholtz_fields(c0, rho, T(d["alpha"]), T(d["sources"]), d["dx"], d["omega"], d["nabs"], d["gamma_max"],
                            precision="fp64", tol=1e-12)
    J = AG.receiver_misfit(f, data, rec)
    J.backward()
    # oracle: forward + adjoint Born solves in float64 on the host, the same misfit, the gradient formula
    P = O.Problem(d["c0"], d["rho"], d["alpha"], d["dx"], d["omega"], d["nabs"], d["gamma_max"])
    src = d["sources"]
    fields = np.stack([P.solve_field(s_, 1e-12, check_every=25, nu=0.8)[0] for s_ in src])
    Jo, g = OG.receiver_misfit(fields, data_h, d["receivers"])
    adj = np.stack([P.unscale(P.solve(P.scale_source(gs, adjoint=True), 1e-12, check_every=25, nu=0.8,
                                      adjoint=True)[0]) for gs in g])
    gc, gr = OG.medium_gradient(d["c0"], d["rho"], d["alpha"], d["omega"], d["nabs"], d["gamma_max"], src, fields,
                                adj)
    assert abs(J.item() - Jo) <= 1e-9 * Jo
    assert np.linalg.norm(c0.grad.cpu().numpy() - gc) <= 1e-8 * np.linalg.norm(gc)
    assert np.linalg.norm(rho.grad.cpu().numpy() - gr) <= 1e-8 * np.linalg.norm(gr)


def _fd_check(n, n_abs, n_vox, tol_solve, rel_tol):
    """Central differences (relative step h = 1e-4) of the misfit at n_vox seeded interior voxels, alternating
    c0 and rho, against the autograd gradient.  Each perturbed misfit solves every source again from the
    unperturbed field (x0), to the same residual tolerance."""
    from paper_2507_16087_gb300 import autograd as AG, cbs

    d = _problem(n, n_abs)
    data, rec = _data(d, "fp32_refine", tol_solve)
    kw = dict(precision="fp32_refine", tol=tol_solve)
    c0 = T(d["c0"]).requires_grad_(True)
    rho = T(d["rho"]).requires_grad_(True)
    src, alpha = T(d["sources"]), T(d["alpha"])
    f = AG.helmholtz_fields(c0, rho, alpha, src, d["dx"], d["omega"], d["nabs"], d["gamma_max"], **kw)
    J = AG.receiver_misfit(f, data, rec)
    J.backward()
    gc, gr = c0.grad.cpu().numpy(), rho.grad.cpu().numpy()
    base = f.detach()

    def Jat(cc, rr):
        s = cbs.solver_create(T(cc), T(rr), alpha, d["dx"], d["omega"], d["nabs"], d["gamma_max"], **kw)
        ff = torch.empty_like(base)
        for k in range(base.shape[0]):
            s.solve_forward(src[k], ff[k], x0=base[k].clone())
        s.destroy()
        return AG.receiver_misfit(ff, data, rec).item()

    h = 1e-4
    worst = 0.0
    for k, (iz, iy, ix) in enumerate(d["fd_voxels"][:n_vox]):
        which = "c0" if k % 2 == 0 else "rho"
        bm = d["c0"] if which == "c0" else d["rho"]
        m = bm[iz, iy, ix]
        mp, mm = bm.copy(), bm.copy()
        mp[iz, iy, ix] = m * (1 + h)
        mm[iz, iy, ix] = m * (1 - h)
        if which == "c0":
            fd = (Jat(mp, d["rho"]) - Jat(mm, d["rho"])) / (2 * h * m)
            g = gc[iz, iy, ix]
        else:
            fd = (Jat(d["c0"], mp) - Jat(d["c0"], mm)) / (2 * h * m)
            g = gr[iz, iy, ix]
        err = abs(g - fd) / max(abs(fd), 1e-30)
        worst = max(worst, err)
        assert err <= rel_tol, (which, (iz, iy, ix), g, fd, err)
    print(f"central differences at {n_vox} voxels of {n}^3: worst relative error {worst:.2e}")
    return worst, gc, gr, d, data, rec


def test_gradient_central_differences_64():
    _fd_check(64, 10, 10, 1e-12, 1e-3)


def test_gradient_central_differences_128_and_checkpointing():
    """The layered-inversion workload at its full size (128^3, 8 sources, 64 receivers): central differences
    at 20 voxels within 1e-3; the checkpointed backward gives the stored-field gradient."""
    from paper_2507_16087_gb300 import autograd as AG

    worst, gc, gr, d, data, rec = _fd_check(128, 20, 20, 1e-12, 1e-3)
    # the recomputing (checkpointed) backward gives the same gradient
    c0 = T(d["c0"]).requires_grad_(True)
    rho = T(d["rho"]).requires_grad_(True)
    f = AG.helmholtz_fields(c0, rho, T(d["alpha"]), T(d["sources"]), d["dx"], d["omega"], d["nabs"], d["gamma_max"],
                            precision="fp32_refine", tol=1e-12, checkpoint=True)
    AG.receiver_misfit(f, data, rec).backward()
    assert np.linalg.norm(c0.grad.cpu().numpy() - gc) <= 1e-9 * np.linalg.norm(gc)
    assert np.linalg.norm(rho.grad.cpu().numpy() - gr) <= 1e-9 * np.linalg.norm(gr)
