"""The oracle's pins catch plausible mistakes in it.

Each mutant below is a copy of the oracle's C source with one planted slip of the kind the pins are meant to catch:
a dropped term, a flipped sign, a wrong index, a transposed operand.  The copy is compiled on the CPU into a
library of its own, and the oracle's pin tests run against it in a child process (the oracle loader takes the copy's
paths from CBS_ORACLE_SRC / CBS_ORACLE_LIB there); at least one pin must fail for every mutant.  The oracle's own
source and library are never touched, and no GPU code is involved.
"""
import concurrent.futures as cf
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "cbs_oracle.c")
# fast pin files first; a child stops at its first failure
PINS = ["tests/test_oracle_operators.py", "tests/test_oracle_solve.py", "tests/test_oracle_fft.py",
        "tests/test_oracle_gradient.py"]

# (what the slip is and which passage it breaks, exact text in the oracle, planted text)
MUTANTS = [
    ("complex sound speed with the absorption term's sign flipped (eq. 118)",
     "c0[i] * c0[i] / (1.0 - 2.0 * I * alpha[i] * c0[i] / omega)",
     "c0[i] * c0[i] / (1.0 + 2.0 * I * alpha[i] * c0[i] / omega)"),
    ("staggered density taken at the cell itself instead of the two-point mean (App. B.1)",
     "0.5 * (rho[i] + rho[neighbour_plus(i, eta, ndim, n)])",
     "rho[i]"),
    ("velocity diagonal without the absorbing layer: S+ rho * i omega (App. B.1)",
     "d[eta * N + i] = rs * (gs + I * omega);",
     "d[eta * N + i] = rs * (I * omega);"),
    ("pressure diagonal with rho c^2 multiplied instead of divided (eq. HH1stOrderSH)",
     "q[i] = (I * omega + g) * P->inv_rho_c2[i];",
     "q[i] = (I * omega + g) / P->inv_rho_c2[i];"),
    ("midrange shift whose imaginary part is taken from the real parts (Algorithm 1 preprocessing)",
     "return 0.5 * (rmin + rmax) + I * 0.5 * (imin + imax);",
     "return 0.5 * (rmin + rmax) + I * 0.5 * (rmin + rmax);"),
    ("lambda = max deviation times beta instead of divided by it (eq. C)",
     "P->lam1 = m1 > 0 ? m1 / beta : cabs(P->a1);",
     "P->lam1 = m1 > 0 ? m1 * beta : cabs(P->a1);"),
    ("pressure block of V scaled by lambda1 (wrong index, eq. LV)",
     "P->v[ndim * N + i] = (q[i] - P->a2) / P->lam2;",
     "P->v[ndim * N + i] = (q[i] - P->a2) / P->lam1;"),
    ("wavenumbers without the negative half of fftfreq",
     "long f = (j < (L + 1) / 2) ? j : j - L;",
     "long f = j;"),
    ("pressure source scaled by lambda1^-1/2 (wrong index, Sec. 2.3.1)",
     "s[D * N + i] * P->inv_rho_c2[i]) * r2;",
     "s[D * N + i] * P->inv_rho_c2[i]) * r1;"),
    ("velocity source without the staggered density (eq. HH1stOrderSH)",
     "P->rho_stag[eta * N + i] * s[eta * N + i]) * r1;",
     "s[eta * N + i]) * r1;"),
    ("(L+I)^-1 without the half-cell shift filters (App. B.1)",
     "S[e] = P->collocated ? 1.0 : cexp(I * kv[e] * P->dx / 2.0);",
     "S[e] = 1.0;"),
    ("(L+I)^-1 diagonal with mu in place of mu - k_eta^2 (dropped term, App. B.1)",
     "G[e][f] = l0 * (mu - kv[e] * kv[e]) / ((a + l0) * mu);",
     "G[e][f] = l0 * mu / ((a + l0) * mu);"),
    ("(L+I)^-1 off-diagonal velocity block with the shifts transposed (App. B.1)",
     "(S[e] * conj(S[f]))",
     "(conj(S[e]) * S[f])"),
    ("(L+I)^-1 pressure row without the conjugate shift (transposed operand, App. B.1)",
     "G[D][e] = -I * kv[e] * sq * conj(S[e]) / mu;",
     "G[D][e] = -I * kv[e] * sq * S[e] / mu;"),
    ("(L+I)^-1 pressure entry with lambda1 for lambda2 (wrong index, App. B.1)",
     "G[D][D] = l1 * (a + l0) / mu;",
     "G[D][D] = l0 * (a + l0) / mu;"),
    ("L symbol's velocity row with the derivative sign flipped (eq. LV)",
     "Lm[e][D] = I * kv[e] * Se / sq;",
     "Lm[e][D] = -I * kv[e] * Se / sq;"),
    ("adjoint apply without the conjugate transpose (M instead of M^H)",
     "(mode >= 2 ? conj(M[c][r]) : M[r][c])",
     "(mode >= 2 ? M[r][c] : M[r][c])"),
    ("A_s x without the potential V x (dropped term, eq. LV)",
     "out[i] += (adjoint ? conj(P->v[i]) : P->v[i]) * x[i];",
     "out[i] += 0.0 * x[i];"),
    ("pre-FFT fuse B x - y (flipped sign, eq. BornAlt)",
     "w[i] = B * x[i] + y[i];",
     "w[i] = B * x[i] - y[i];"),
    ("Born update without B (dropped factor, eq. BornAlt)",
     "cplx delta = nu * B * (z[i] - x[i]);",
     "cplx delta = nu * (z[i] - x[i]);"),
    ("true residual y + A_s x (flipped sign)",
     "r[i] = y[i] - r[i];",
     "r[i] = y[i] + r[i];"),
    ("FFT combination step with the root index missing its stride (own FFT)",
     "acc += tw[((q * k) % n) * step] * scratch[q * m + (k % m)];",
     "acc += tw[(q * k) % n] * scratch[q * m + (k % m)];"),
    ("inverse FFT without the 1/N factor (own FFT)",
     "double s = 1.0 / (double)total;",
     "double s = 1.0;"),
    ("output pressure unscaled by lambda1^-1/2 (wrong index, Algorithm 1 output)",
     "field[D * N + i] = x[D * N + i] * r2;",
     "field[D * N + i] = x[D * N + i] * r1;"),
    ("true residual without the square root",
     "double rr = sqrt(norm2(r, CN) / norm2(y, CN));",
     "double rr = norm2(r, CN) / norm2(y, CN);"),
    ("Algorithm 1's increment not normalised by ||x||",
     "if (incr) incr[it] = xx > 0 ? sqrt(dd / xx) : 0.0;",
     "if (incr) incr[it] = xx > 0 ? sqrt(dd) : 0.0;"),
    ("median of an even count taken as the upper middle value (Algorithm 1's example shift)",
     "return (m % 2) ? v[m / 2] : 0.5 * (v[m / 2 - 1] + v[m / 2]);",
     "return v[m / 2];"),
    ("minimum enclosing circle through two points centred on one of them (Sec. 4)",
     "c = 0.5 * (pi + pj);",
     "c = pi;"),
    ("absorbing layer's inner edge one cell off on the high side",
     "double t = (xi - (double)(N - 1 - n_hi)) / (double)n_hi;",
     "double t = (xi - (double)(N - n_hi)) / (double)n_hi;"),
    ("absorbing layer from the last axis only (gamma summed over axes, Sec. 2.1 reading)",
     "g += layer_axis(xi[a], (long)n[a], nabs + 2 * a, gmax, power);",
     "g = layer_axis(xi[a], (long)n[a], nabs + 2 * a, gmax, power);"),
    ("symbol's mu without lambda2 (dropped term, App. B.1)",
     "const cplx mu = k2 + (a + l0) * (b + l1);",
     "const cplx mu = k2 + (a + l0) * b;"),
    ("adjoint (L+I)^-1 applied as the forward one",
     "fourier_apply(P, in, out, adjoint ? 2 : 0);",
     "fourier_apply(P, in, out, 0);"),
    ("adjoint A_s with V instead of conj(V)",
     "out[i] += (adjoint ? conj(P->v[i]) : P->v[i]) * x[i];",
     "out[i] += P->v[i] * x[i];"),
    ("adjoint fuse with B instead of conj(B)",
     "cplx B = 1.0 - (adjoint ? conj(P->v[i]) : P->v[i]);\n            w[i] = B * x[i] + y[i];",
     "cplx B = 1.0 - P->v[i];\n            w[i] = B * x[i] + y[i];"),
    ("solve loop stopping at ten times the tolerance",
     "while (r > tol && it < max_iter) {",
     "while (r > 10.0 * tol && it < max_iter) {"),
]


def _run_mutant(k, tmp):
    """Plant mutant k (k < 0: the unchanged source, as a control), build it, run the pins on it in a child.
    Returns (pytest exit code, first failing test, output tail)."""
    src = open(SRC).read()
    mutant = src if k < 0 else src.replace(MUTANTS[k][1], MUTANTS[k][2])
    tag = "control" if k < 0 else f"mutant{k}"
    path = os.path.join(tmp, f"{tag}.c")
    lib = os.path.join(tmp, f"lib{tag}.so")
    with open(path, "w") as f:
        f.write(mutant)
    # built here, so that a child's failure is a pin's verdict and never a build error
    b = subprocess.run(["gcc", "-O2", "-std=c99", "-fopenmp", "-fPIC", "-shared", path, "-o", lib, "-lm"],
                       capture_output=True, text=True)
    assert b.returncode == 0, (tag, b.stderr[-600:])
    env = dict(os.environ, CBS_ORACLE_SRC=path, CBS_ORACLE_LIB=lib, OMP_NUM_THREADS="2")
    r = subprocess.run([sys.executable, "-m", "pytest", *PINS, "-x", "-q", "-m", "not gpu", "-p", "no:cacheprovider"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    out = r.stdout + r.stderr
    first = next((ln.split()[1] for ln in out.splitlines() if ln.startswith("FAILED ")), "")
    return r.returncode, first, out[-600:]


def test_mutants_are_well_defined():
    src = open(SRC).read()
    for desc, old, new in MUTANTS:
        assert src.count(old) == 1, desc       # each slip is planted at exactly one place
        assert old != new


def test_every_planted_mistake_fails_a_pin(tmp_path):
    workers = max(1, min(6, (os.cpu_count() or 2) // 2))
    with cf.ThreadPoolExecutor(max_workers=workers) as ex:
        results = list(ex.map(lambda k: _run_mutant(k, str(tmp_path)), range(-1, len(MUTANTS))))
    control, results = results[0], results[1:]
    assert control[0] == 0, control[2]        # the harness itself passes the unchanged oracle
    survivors = [(MUTANTS[k][0], out) for k, (rc, _, out) in enumerate(results) if rc == 0]
    assert not survivors, survivors
    # a child that could not collect or was interrupted (pytest exit codes 2-4) would not have tested the pins
    for k, (rc, first, out) in enumerate(results):
        assert rc == 1 and first, (MUTANTS[k][0], rc, out)
        print(f"{MUTANTS[k][0]}: {first}")


# the gradient oracle (oracle/gradient.py, Sec. 2.3's adjoint-state formula) against its finite-difference pin
GRAD_SRC = os.path.join(ROOT, "oracle", "gradient.py")
GRAD_MUTANTS = [
    ("d(c^2)/dc0 factor with the wrong sign on its real part", "fac = -2.0 / c0 ** 3", "fac = 2.0 / c0 ** 3"),
    ("staggered density's second neighbour dropped", "np.real(term + np.roll(term, 1, axis=ax))",
     "np.real(term)"),
    ("staggered density's second neighbour on the wrong side", "np.roll(term, 1, axis=ax)",
     "np.roll(term, -1, axis=ax)"),
    ("adjoint field not conjugated in the c0 term", "grad_c += np.real(np.conj(lp) *", "grad_c += np.real(lp *"),
    ("dq/drho with the wrong sign", "(-bp / rho + q / rho * p)", "(-bp / rho - q / rho * p)"),
    ("misfit without its factor 1/2 (adjoint source no longer its derivative)",
     "J = 0.5 * float(np.sum(np.abs(r) ** 2))", "J = float(np.sum(np.abs(r) ** 2))"),
    ("staggered layer values taken at the cell centres in the density derivative",
     "stag.append(dense.layer_profile(n, nabs[a][0], nabs[a][1], gamma_max, power, 0.5).reshape(sh))",
     "stag.append(dense.layer_profile(n, nabs[a][0], nabs[a][1], gamma_max, power, 0.0).reshape(sh))"),
]


def _gradient_module(text):
    import types

    mod = types.ModuleType("oracle.gradient_planted")
    mod.__package__ = "oracle"
    exec(compile(text, GRAD_SRC, "exec"), mod.__dict__)
    return mod


def test_planted_mistakes_in_the_gradient_oracle_fail_its_pin(monkeypatch):
    import test_oracle_gradient as TG

    src = open(GRAD_SRC).read()

    def pin_fails(text):
        monkeypatch.setattr(TG, "gradient", _gradient_module(text))
        try:
            for which in ("c0", "rho"):
                TG.test_gradient_matches_central_differences_dense(which)
        except AssertionError:
            return True
        return False

    assert not pin_fails(src)                   # control: the unchanged formula passes the pin
    for desc, old, new in GRAD_MUTANTS:
        assert src.count(old) == 1, desc
        assert pin_fails(src.replace(old, new)), desc


# the Python parts of the oracle, planted in a child process by a plugin that loads a slipped copy of the module
# (oracle.dense: the discrete system assembled densely; oracle.analytic: the free-space and series fields) before
# the pins import it
_PLUGIN = '''import importlib.util, os, sys
import oracle
_name = os.environ["CBS_PLANTED_MODULE"]
_spec = importlib.util.spec_from_file_location(_name, os.environ["CBS_PLANTED_PATH"])
_mod = importlib.util.module_from_spec(_spec)
sys.modules[_name] = _mod
_spec.loader.exec_module(_mod)
setattr(oracle, _name.split(".")[1], _mod)
'''


def _run_module_mutant(module, src_path, pins, text, tag, tmp, select=()):
    path = os.path.join(tmp, f"{tag}.py")
    with open(path, "w") as f:
        f.write(text)
    with open(os.path.join(tmp, "planted_module_plugin.py"), "w") as f:
        f.write(_PLUGIN)
    env = dict(os.environ, CBS_PLANTED_MODULE=module, CBS_PLANTED_PATH=path, OMP_NUM_THREADS="2",
               PYTHONPATH=os.pathsep.join([tmp, ROOT, os.environ.get("PYTHONPATH", "")]))
    r = subprocess.run([sys.executable, "-m", "pytest", *pins, *select, "-x", "-q", "-m", "not gpu", "-p",
                        "no:cacheprovider", "-p", "planted_module_plugin"], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=900)
    out = r.stdout + r.stderr
    first = next((ln.split()[1] for ln in out.splitlines() if ln.startswith("FAILED ")), "")
    return r.returncode, first, out[-600:]


def _check_module_mutants(module, src_path, pins, mutants, tmp, select=()):
    src = open(src_path).read()
    for desc, old, new in mutants:
        assert src.count(old) == 1, desc
    texts = [src] + [src.replace(old, new) for _, old, new in mutants]
    tags = [f"{module.split('.')[1]}_control"] + [f"{module.split('.')[1]}{k}" for k in range(len(mutants))]
    workers = max(1, min(6, (os.cpu_count() or 2) // 2))
    with cf.ThreadPoolExecutor(max_workers=workers) as ex:
        results = list(ex.map(lambda k: _run_module_mutant(module, src_path, pins, texts[k], tags[k], tmp, select),
                              range(len(texts))))
    control, results = results[0], results[1:]
    assert control[0] == 0, control[2]
    for k, (rc, first, out) in enumerate(results):
        assert rc == 1 and first, (mutants[k][0], rc, out)
        print(f"{mutants[k][0]}: {first}")


DENSE_MUTANTS = [
    ("complex sound speed with the absorption term's sign flipped (eq. 118)",
     "    c2 = c0 ** 2 / (1 - 2j * alpha * c0 / omega)\n    per_axis_c = []",
     "    c2 = c0 ** 2 / (1 + 2j * alpha * c0 / omega)\n    per_axis_c = []"),
    ("staggered density averaged with the neighbour on the wrong side (App. B.1)",
     "np.roll(rho, -1, axis=D - 1 - eta)", "np.roll(rho, 1, axis=D - 1 - eta)"),
    ("forward staggered derivative with the backward half-cell shift (App. B.1)",
     "dplus = Fi @ np.diag(1j * k * np.exp(1j * k * sh)) @ F",
     "dplus = Fi @ np.diag(1j * k * np.exp(-1j * k * sh)) @ F"),
    ("velocity rows coupled through the backward derivative (transposed blocks)",
     "A[eta * N:(eta + 1) * N, D * N:] = axis_operator(shape, eta, dplus)",
     "A[eta * N:(eta + 1) * N, D * N:] = axis_operator(shape, eta, dminus)"),
    ("velocity source without the staggered density (eq. HH1stOrderSH)",
     "out[eta] = rho_s[eta] * src[eta]", "out[eta] = src[eta]"),
    ("absorbing layer evaluated at the cell centres for the staggered points (App. B.1)",
     "0.0 if collocated else 0.5", "0.0"),
    ("wavenumbers without the negative half of fftfreq",
     "f = np.array([j if j < (n + 1) // 2 else j - n for j in range(n)], dtype=np.float64)",
     "f = np.array([j for j in range(n)], dtype=np.float64)"),
    ("pressure diagonal without the absorbing layer (eq. HH1stOrderSH)",
     "q = (1j * omega + gamma) / (rho * c2)\n    d = []", "q = (1j * omega) / (rho * c2)\n    d = []"),
]


def test_planted_mistakes_in_the_plain_definition_fail_a_pin(tmp_path):
    _check_module_mutants("oracle.dense", os.path.join(ROOT, "oracle", "dense.py"),
                          ["tests/test_oracle_operators.py", "tests/test_oracle_solve.py"], DENSE_MUTANTS, str(tmp_path))


ANALYTIC_MUTANTS = [
    ("spherical Hankel function of the first kind (the wrong time convention)",
     "special.spherical_jn(m, z, derivative=derivative) - 1j * special.spherical_yn(m, z, derivative=derivative)",
     "special.spherical_jn(m, z, derivative=derivative) + 1j * special.spherical_yn(m, z, derivative=derivative)"),
    ("3D point source normalised by dx^2 instead of dx^3",
     "(1j * omega * S * dx ** 3 / c ** 2) * np.exp(-1j * k * R) / (4 * np.pi * R)",
     "(1j * omega * S * dx ** 2 / c ** 2) * np.exp(-1j * k * R) / (4 * np.pi * R)"),
    ("2D Green's function with +i/4 instead of -i/4",
     "(1j * omega * S * dx ** 2 / c ** 2) * (-0.25j) * H2(0, k * R)",
     "(1j * omega * S * dx ** 2 / c ** 2) * (0.25j) * H2(0, k * R)"),
    ("sphere monopole coefficient at the sphere radius instead of the source distance (App. C reading)",
     "        L = amp * (-1j * k0 / (4 * np.pi)) * h2(m, k0 * r_s)\n        M = np.array",
     "        L = amp * (-1j * k0 / (4 * np.pi)) * h2(m, k0 * a)\n        M = np.array"),
    ("disc interior velocity with the exterior impedance (App. C)",
     "-special.jvp(m, k1 * a) / Z1]", "-special.jvp(m, k1 * a) / Z0]"),
    ("disc plane-wave expansion without the Neumann factor",
     "        inc = (1.0 if m == 0 else 2.0) * (-1j) ** m\n", "        inc = (-1j) ** m\n"),
    ("scatterer's complex sound speed with the absorption term's sign flipped (eq. 118)",
     "np.sqrt(c0 ** 2 / (1 - 2j * alpha * c0 / omega))", "np.sqrt(c0 ** 2 / (1 + 2j * alpha * c0 / omega))"),
]


def test_planted_mistakes_in_the_analytic_fields_fail_a_pin(tmp_path):
    # the two slow refinement studies (1-D interface, disc) are left out: the series and point-source pins decide
    _check_module_mutants("oracle.analytic", os.path.join(ROOT, "oracle", "analytic.py"),
                          ["tests/test_oracle_physics.py"], ANALYTIC_MUTANTS, str(tmp_path),
                          select=("-k", "not reflection_coefficient and not disc_scattering"))
