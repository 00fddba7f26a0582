"""Compile-time FFT plans of the CUDA engine (csrc/fft.cuh) for every (length, values-per-thread) pair the
launchers (csrc/launch.cuh) choose, checked on the host: the pass radices multiply to the length and divide
the thread's value count, each pass's slot order is a permutation with q_slot its inverse, and the twiddle
cache holds exactly the twiddles the passes use.  CPU test (nvcc compiles the plan functions for the host)."""
import ctypes
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2507_16087_gb300", "csrc")
SIZES = [8, 12, 16, 24, 32, 48, 64, 96, 128, 192, 256, 512, 1024, 2048]

SRC = r'''
#include "launch.cuh"
using namespace cbs;

// values per thread chosen by the launchers for extent n
extern "C" void r_choices(int n, int* out) {
    out[0] = r_rows<float>(n);  out[1] = r_rows<double>(n);
    out[2] = r_axis<float>(n);  out[3] = r_axis<double>(n);
    out[4] = r_last<float>(n, 4);  out[5] = r_last<double>(n, 4);
    out[6] = r_tile<float>(n);     out[7] = r_last<float>(n, 3);  out[8] = r_last<double>(n, 3);
}
extern "C" int npass(int n, int r) { return plan_npass(n, r); }
extern "C" int radix(int n, int r, int p) { return plan_radix(n, r, p); }
extern "C" int twcount(int n, int r) { return tw_count(n, r); }

template <int N, int R, int P> void fill_p(int* sq, int* qs) {
    constexpr int np = plan_npass(N, R);
    if constexpr (P <= np) {
        for (int s = 0; s < R; ++s) { sq[P * R + s] = slot_q<N, R, P>(s); qs[P * R + s] = q_slot<N, R, P>(s); }
        fill_p<N, R, P + 1>(sq, qs);
    }
}
template <int N, int R> int fill(int* sq, int* qs) {
    if constexpr (N % R != 0 || plan_npass(N, R) <= 0) return -1;
    else { fill_p<N, R, 0>(sq, qs); return plan_npass(N, R); }
}
#define CASE_R(N) \
    if (r == 4) return fill<N, 4>(sq, qs); if (r == 6) return fill<N, 6>(sq, qs); \
    if (r == 8) return fill<N, 8>(sq, qs); if (r == 12) return fill<N, 12>(sq, qs); \
    if (r == 16) return fill<N, 16>(sq, qs); if (r == 24) return fill<N, 24>(sq, qs); return -2;
extern "C" int slots(int n, int r, int* sq, int* qs) {
    switch (n) {
#define CBS_CASE(N) case N: { CASE_R(N) }
        CBS_FOR_EACH_SIZE(CBS_CASE)
#undef CBS_CASE
    }
    return -3;
}
'''


@pytest.fixture(scope="module")
def lib():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    d = tempfile.mkdtemp()
    src = os.path.join(d, "plans.cu")
    open(src, "w").write(SRC)
    so = os.path.join(d, "plans.so")
    subprocess.check_call([nvcc, "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a", "-Xcompiler", "-fPIC",
                           "-shared", "-I" + CSRC, "-I" + os.path.join(ROOT, "include"), src, "-o", so])
    L = ctypes.CDLL(so)
    for f in ("npass", "twcount"):
        getattr(L, f).argtypes = [ctypes.c_int, ctypes.c_int]
    L.radix.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int]
    L.r_choices.argtypes = [ctypes.c_int, ctypes.c_void_p]
    L.slots.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    return L


def _pairs(L):
    out = set()
    for n in SIZES:
        rc = np.zeros(9, dtype=np.int32)
        L.r_choices(n, rc.ctypes.data)
        out |= {(n, int(r)) for r in rc}
        if n in (32, 64, 128):
            out.add((n, 8))  # plane kernels
    return sorted(out)


def test_every_chosen_plan_factors_the_length(lib):
    for n, r in _pairs(lib):
        if r > n:
            continue  # a value count above the length is never launched for that extent
        npass = lib.npass(n, r)
        assert npass > 0, (n, r)
        rad = [lib.radix(n, r, p) for p in range(npass)]
        assert int(np.prod(rad)) == n, (n, r, rad)
        assert all(x in (2, 3, 4, 8, 16) and r % x == 0 for x in rad), (n, r, rad)


def test_slot_orders_are_permutations_with_inverses(lib):
    for n, r in _pairs(lib):
        if r > n:
            continue
        sq = np.full(32 * r, -1, dtype=np.int32)
        qs = np.full(32 * r, -1, dtype=np.int32)
        npass = lib.slots(n, r, sq.ctypes.data, qs.ctypes.data)
        assert npass == lib.npass(n, r), (n, r)
        for p in range(npass + 1):
            a, b = sq[p * r:(p + 1) * r], qs[p * r:(p + 1) * r]
            assert sorted(a) == list(range(r)), (n, r, p)
            assert all(b[a[s]] == s for s in range(r)), (n, r, p)


def test_twiddle_count_matches_the_passes(lib):
    # pass p with ns = product of the earlier radices > 1 multiplies inputs 1..radix-1 of each of the thread's
    # r / radix butterflies by a twiddle
    for n, r in _pairs(lib):
        if r > n:
            continue
        npass = lib.npass(n, r)
        ns, count = 1, 0
        for p in range(npass):
            x = lib.radix(n, r, p)
            if ns > 1:
                count += (r // x) * (x - 1)
            ns *= x
        assert lib.twcount(n, r) == count, (n, r)
