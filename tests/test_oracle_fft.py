"""Pins of the oracle's own FFT (a library special case: numpy.fft)."""
import numpy as np
import pytest

import oracle

SIZES_1D = [1, 2, 3, 4, 5, 6, 7, 8, 9, 11, 12, 13, 15, 16, 17, 20, 24, 25, 27,
            30, 32, 45, 60, 64, 96, 97, 100, 125, 128, 160, 256]


@pytest.mark.parametrize("n", SIZES_1D)
def test_fft1d_matches_numpy(n):
    rng = np.random.default_rng(n)
    a = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    ref = np.fft.fft(a)
    got = oracle.fft1d(a, -1)
    assert np.max(np.abs(got - ref)) <= 1e-12 * max(1.0, np.max(np.abs(ref)))
    inv = oracle.fft1d(a, +1)
    assert np.allclose(inv, np.fft.ifft(a) * n, rtol=0, atol=1e-12 * n)


@pytest.mark.parametrize("shape", [(4, 4, 4), (5, 6, 7), (8, 3, 10), (16, 16, 16),
                                   (1, 9, 12), (24, 20, 18)])
def test_fft3d_matches_numpy_and_roundtrips(shape):
    rng = np.random.default_rng(sum(shape))
    a = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    F = oracle.fft3d(a, -1)
    assert np.max(np.abs(F - np.fft.fftn(a))) <= 1e-11 * np.max(np.abs(F))
    back = oracle.fft3d(F, +1) / a.size
    assert np.max(np.abs(back - a)) <= 1e-13 * 10 * np.log2(a.size + 1)
