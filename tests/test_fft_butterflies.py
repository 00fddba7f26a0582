"""The r-point DFT butterflies of the CUDA FFT engine (csrc/fft.cuh), compiled
for the host with nvcc, against numpy's FFT (CPU test; no GPU needed)."""
import ctypes
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2507_16087_gb300", "csrc")

SRC = r'''
#include "fft.cuh"
using namespace cbs;
template <int r, int S> static void run(const double* in, double* out) {
    double2 v[r];
    for (int i = 0; i < r; ++i) v[i] = make_double2(in[2 * i], in[2 * i + 1]);
    dft<r, S>(v);
    for (int i = 0; i < r; ++i) { out[2 * i] = v[i].x; out[2 * i + 1] = v[i].y; }
}
extern "C" int butterfly(int r, int s, const double* in, double* out) {
    if (s < 0) {
        switch (r) { case 2: run<2, -1>(in, out); return 0; case 3: run<3, -1>(in, out); return 0;
                     case 4: run<4, -1>(in, out); return 0; case 8: run<8, -1>(in, out); return 0;
                     case 16: run<16, -1>(in, out); return 0; }
    } else {
        switch (r) { case 2: run<2, 1>(in, out); return 0; case 3: run<3, 1>(in, out); return 0;
                     case 4: run<4, 1>(in, out); return 0; case 8: run<8, 1>(in, out); return 0;
                     case 16: run<16, 1>(in, out); return 0; }
    }
    return 1;
}
'''


@pytest.fixture(scope="module")
def lib():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    d = tempfile.mkdtemp()
    src = os.path.join(d, "bf.cu")
    open(src, "w").write(SRC)
    so = os.path.join(d, "bf.so")
    subprocess.check_call([nvcc, "-std=c++17", "-Xcompiler", "-fPIC", "-shared", "-I" + CSRC, src, "-o", so])
    L = ctypes.CDLL(so)
    L.butterfly.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    return L


@pytest.mark.parametrize("r", [2, 3, 4, 8, 16])
@pytest.mark.parametrize("s", [-1, 1])
def test_butterfly_is_the_dft(lib, r, s):
    rng = np.random.default_rng(r)
    x = rng.standard_normal(r) + 1j * rng.standard_normal(r)
    out = np.zeros(r, dtype=np.complex128)
    assert lib.butterfly(r, s, x.ctypes.data, out.ctypes.data) == 0
    ref = np.fft.fft(x) if s < 0 else np.fft.ifft(x) * r
    assert np.max(np.abs(out - ref)) <= 1e-14 * r
