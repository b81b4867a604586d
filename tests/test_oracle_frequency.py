"""Pins of the frequency vectors, eqs. (freq) and (freqrot)."""
import itertools

import numpy as np
import pytest

import oracle


def q_of(k, n):
    m = k if 2 * k < n else k - n
    return 2 * np.pi * m / n


@pytest.mark.parametrize("shape", [(8, 8, 8), (6, 10, 7), (5, 5, 5)])
def test_rotated_equals_tan_form_off_nyquist(shape):
    """xi'_p = i 2 N_p tan(q_p/2) prod_r 1/2 (1 + e^{i q_r}) as printed in
    eq. (freqrot), with the product over all axes r, wherever tan is finite."""
    for k in itertools.product(*[range(n) for n in shape]):
        q = [q_of(k[p], shape[p]) for p in range(3)]
        if any(abs(abs(qq) - np.pi) < 1e-12 for qq in q):
            continue
        prod = np.prod([0.5 * (1 + np.exp(1j * qq)) for qq in q])
        ref = np.array([1j * 2 * shape[p] * np.tan(q[p] / 2) * prod for p in range(3)])
        got = oracle.frequency(shape, k, 1)
        assert np.allclose(got, ref, rtol=1e-12, atol=1e-12 * max(shape))


def test_continuous_frequency():
    shape = (8, 6, 5)
    for k in [(0, 0, 0), (1, 2, 3), (4, 3, 2), (7, 5, 4)]:
        got = oracle.frequency(shape, k, 0)
        ref = np.array([1j * q_of(k[p], shape[p]) * shape[p] for p in range(3)])
        assert np.allclose(got, ref, rtol=1e-14, atol=1e-13)


def test_rotated_is_symbol_of_real_space_stencil():
    """Brute force: the rotated forward difference (edge-averaged over the
    2x2x2 voxel cube) applied to the plane wave exp(2 pi i k.n/N) returns
    xi' times the wave (forward DFT sign exp(-2 pi i k n / N))."""
    shape = (6, 5, 4)
    rng = np.random.default_rng(0)
    grid = np.meshgrid(*[np.arange(n) for n in shape], indexing="ij")
    for _ in range(12):
        k = tuple(int(rng.integers(0, n)) for n in shape)
        wave = np.exp(2j * np.pi * sum(k[p] * grid[p] / shape[p] for p in range(3)))
        xi = oracle.frequency(shape, k, 1)
        for p in range(3):
            others = [r for r in range(3) if r != p]
            acc = np.zeros(shape, dtype=complex)
            for c in itertools.product([0, 1], repeat=2):
                shift = [0, 0, 0]
                for r, cr in zip(others, c):
                    shift[r] = cr
                base = np.roll(wave, [-s for s in shift], axis=(0, 1, 2))
                fwd = np.roll(base, -1, axis=p)
                acc += fwd - base
            deriv = shape[p] * acc / 4.0
            assert np.allclose(deriv, xi[p] * wave, atol=1e-11)
