"""Pins for the oracle's own FFT: the DFT sum itself on small sizes, numpy.fft
as a library special case, Parseval and the round trip."""
import numpy as np
import pytest

from oracle import oracle as O


def naive_dft(x, sign=-1):
    n = len(x)
    j = np.arange(n)
    # the definition X_k = sum_j x_j exp(sign 2 pi i j k / n), summed term by term
    out = np.zeros(n, dtype=np.complex128)
    for k in range(n):
        out[k] = np.sum(x * np.exp(sign * 2j * np.pi * j * k / n))
    return out


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6, 7, 8, 9, 12, 16, 18, 24, 27, 32, 48, 64])
def test_fft1d_matches_dft_sum(n):
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    ref = naive_dft(x)
    got = O.fft1d(x)
    assert np.max(np.abs(got - ref)) <= 1e-13 * max(1.0, np.max(np.abs(ref))) * np.log2(max(n, 2))
    got_inv = O.fft1d(x, +1)
    ref_inv = naive_dft(x, +1)
    assert np.max(np.abs(got_inv - ref_inv)) <= 1e-13 * max(1.0, np.max(np.abs(ref_inv))) * np.log2(max(n, 2))


@pytest.mark.parametrize("n", [64, 96, 128, 192, 512, 1024, 2048])
def test_fft1d_matches_numpy(n):
    rng = np.random.default_rng(n + 1)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    ref = np.fft.fft(x)
    err = np.max(np.abs(O.fft1d(x) - ref)) / np.max(np.abs(ref))
    assert err <= 1e-14 * np.log2(n) * 4


@pytest.mark.parametrize("shape", [(8,), (6, 10), (16, 12), (4, 6, 8), (12, 9, 16)])
def test_fftn_matches_numpy_and_round_trip(shape):
    rng = np.random.default_rng(sum(shape))
    x = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    X = O.fftn(x)
    assert np.allclose(X, np.fft.fftn(x), rtol=0, atol=1e-12 * np.abs(X).max())
    back = O.fftn(X, +1)
    assert np.max(np.abs(back - x)) <= 1e-13 * np.abs(x).max() * 10
    # Parseval: sum |x|^2 = sum |X|^2 / N
    assert np.isclose(np.sum(np.abs(x) ** 2), np.sum(np.abs(X) ** 2) / x.size, rtol=1e-13)


def test_fft_shift_theorem():
    # a shift by one sample multiplies the DFT by exp(-2 pi i k / n)
    n = 48
    rng = np.random.default_rng(5)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    X = O.fft1d(x)
    Xs = O.fft1d(np.roll(x, 1))
    k = np.arange(n)
    assert np.allclose(Xs, X * np.exp(-2j * np.pi * k / n), atol=1e-12)
