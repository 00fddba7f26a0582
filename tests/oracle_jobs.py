"""Long FP64 oracle computations that GPU tests compare against.

TEST INFRASTRUCTURE.  Each job needs only seeded synthetic inputs (workloads,
the oracle itself), never a result of the CUDA path, so it can run in a
background process while the GPU tests run; ``tests/conftest.py`` starts such
processes (fresh interpreters) when a test that needs a job is selected,
and the ``oracle_job`` fixture waits for the job's file.  The jobs of one group
of ``GROUPS`` run one after the other; the groups run side by side.

  sphere128   the 128^3 sphere workload solved to a scaled residual of 1e-8
              (Algorithm 1, nu = 0.8): the reference for the FP32 + FP64
              refinement solve at full size.
  served      two serving-stream requests (64^3 and 512^2 random smooth media
              generated on the host) solved to 1e-9: the references of the same
              requests served in a mix.
  gradient64  the layered-inversion medium at 64^3 (one source, 64 receivers,
              seeded synthetic receiver data): the misfit gradient with respect
              to c0 and rho from forward and adjoint oracle solves (App. B.1
              adjoint, Sec. 2.3) and the adjoint-state formula.
"""
from __future__ import annotations

import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# jobs in one group run one after the other in one background interpreter; the groups run side by side
GROUPS = (("sphere128",), ("gradient64", "served"))

# the two served requests: (rid, numpy shape, medium seed, source (x, y[, z]), PPW, frequency)
SERVED = ((1000, (64, 64, 64), 71, (30, 25, 40), 6.5, 5e5),
          (1001, (512, 512), 72, (100, 300), 5.0, 1e6))

GRAD64 = dict(n=64, n_abs=10, src_grid=(1, 1), rec_grid=(8, 8), data_seed=64, tol=1e-9)


def served_medium(shape, seed, ppw, f_hz):
    from paper_2507_16087_gb300 import workloads as W

    return W.smooth_random_medium(shape, seed=seed, c_range=(1400.0, 2800.0), rho_range=(900.0, 1900.0),
                                  alpha_db_range=(0.0, 5.0), sigma_frac=1.0 / 16, ppw=ppw, n_abs=16, f_hz=f_hz)


def gradient64_inputs():
    """The layered-inversion workload at 64^3 with one source and seeded synthetic receiver data."""
    from paper_2507_16087_gb300 import workloads as W

    g = GRAD64
    d = W.layered_inversion(n=g["n"], n_abs=g["n_abs"], src_grid=g["src_grid"], rec_grid=g["rec_grid"])
    rng = np.random.default_rng(g["data_seed"])
    S, nr = d["sources"].shape[0], d["receivers"][0].size
    d["data"] = 1e-3 * (rng.standard_normal((S, nr)) + 1j * rng.standard_normal((S, nr)))
    return d


def _sphere128():
    from oracle import oracle as O
    from paper_2507_16087_gb300 import workloads as W

    p = W.sphere_128()
    P = O.Problem(p.c0, p.rho, p.alpha, p.dx, p.omega, p.nabs, p.gamma_max)
    f, it, res = P.solve_field(p.source, 1e-8, check_every=100, nu=0.8)
    return {"field": f, "iters": it, "residual": res}


def _served():
    from oracle import oracle as O
    from paper_2507_16087_gb300 import workloads as W

    out = {}
    for rid, shape, seed, pos, ppw, f_hz in SERVED:
        h = served_medium(shape, seed, ppw, f_hz)
        P = O.Problem(h.c0, h.rho, h.alpha, h.dx, h.omega, h.nabs, h.gamma_max)
        f, it, res = P.solve_field(W.point_source(shape, pos), 1e-9, check_every=100, nu=0.8)
        out[f"p{rid}"] = f[len(shape)]
        out[f"res{rid}"] = res
        out[f"iters{rid}"] = it
    return out


def _gradient64():
    from oracle import gradient as OG
    from oracle import oracle as O

    d = gradient64_inputs()
    tol = GRAD64["tol"]
    P = O.Problem(d["c0"], d["rho"], d["alpha"], d["dx"], d["omega"], d["nabs"], d["gamma_max"])
    src = d["sources"]
    fields = np.stack([P.solve_field(s_, tol, check_every=100, nu=0.8)[0] for s_ in src])
    J, g = OG.receiver_misfit(fields, d["data"], d["receivers"])
    adj = np.stack([P.unscale(P.solve(P.scale_source(gs, adjoint=True), tol, check_every=100, nu=0.8,
                                      adjoint=True)[0]) for gs in g])
    gc, gr = OG.medium_gradient(d["c0"], d["rho"], d["alpha"], d["omega"], d["nabs"], d["gamma_max"], src, fields,
                                adj)
    return {"J": J, "grad_c0": gc, "grad_rho": gr}


JOBS = {"sphere128": _sphere128, "served": _served, "gradient64": _gradient64}


def job_path(outdir, name):
    return os.path.join(outdir, name + ".npz")


def main(outdir, names):
    for name in names:
        t0 = time.perf_counter()
        out = JOBS[name]()
        out["seconds"] = time.perf_counter() - t0
        tmp = job_path(outdir, name) + ".tmp.npz"
        np.savez(tmp, **out)
        os.replace(tmp, job_path(outdir, name))
        print(f"oracle job {name}: {out['seconds']:.1f} s", flush=True)


if __name__ == "__main__":
    main(sys.argv[1], sys.argv[2:])
