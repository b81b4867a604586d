"""Pins of the oracle's phase-field smoothening (section 3.2): the filtered
field is the minimiser of the phase-field functional (eq. phase), checked
through its Euler-Lagrange equation with derivatives taken by numpy's FFT (an
independent transform), the mean-density conservation the paper notes, the
limits of zero length and no threshold, and the bounds of a filtered
indicator."""
import numpy as np
import pytest

import oracle
import rve_inputs as ri


def spectral_laplacian(f):
    """periodic Laplacian in units of the voxel, by numpy's FFT"""
    k = [2 * np.pi * np.fft.fftfreq(n) for n in f.shape]
    K2 = k[0][:, None, None] ** 2 + k[1][None, :, None] ** 2 + k[2][None, None, :] ** 2
    return np.real(np.fft.ifftn(-K2 * np.fft.fftn(f)))


@pytest.mark.parametrize("ell,eps", [(1.0, 1.0), (2.5, 1.0), (1.5, 0.3)])
def test_pfs_solves_the_euler_lagrange_equation(ell, eps):
    """ratio 1, no threshold: (l^2/eps) lap(phi) - phi = -omega (eq. phase2)."""
    rng = np.random.default_rng(0)
    omega = (rng.random((12, 10, 14)) > 0.6).astype(float)
    phi = oracle.pfs(omega, 1, ell, eps, threshold=0.0)
    res = (ell ** 2 / eps) * spectral_laplacian(phi) - phi + omega
    assert np.max(np.abs(res)) <= 1e-12


def test_pfs_is_the_minimiser_of_the_functional():
    """E[phi] = sum 1/2 l^2 |grad phi|^2 + eps/2 (phi - omega)^2 grows under
    any perturbation of the filtered field (eq. phase)."""
    ell, eps = 1.3, 1.0
    rng = np.random.default_rng(1)
    omega = (rng.random((10, 10, 10)) > 0.5).astype(float)

    def energy(f):
        return float(np.sum(0.5 * ell ** 2 * (-f * spectral_laplacian(f)) + 0.5 * eps * (f - omega) ** 2))

    phi = oracle.pfs(omega, 1, ell, eps, threshold=0.0)
    e0 = energy(phi)
    for seed in range(5):
        d = np.random.default_rng(10 + seed).standard_normal(phi.shape) * 1e-3
        assert energy(phi + d) > e0 and energy(phi - d) > e0


def test_pfs_conserves_the_mean_density():
    """the filter keeps the xi = 0 term and block averaging keeps the mean
    (section 4 notes the conservation), without threshold"""
    omega, _ = ri.octet(24, 0.15)
    omega = (omega > 0.5).astype(float)
    phi = oracle.pfs(omega, 3, 1.5, threshold=0.0)
    assert phi.shape == (8, 8, 8)
    assert phi.mean() == pytest.approx(omega.mean(), rel=1e-12)


def test_zero_length_is_block_averaging_and_threshold_only_zeroes():
    rng = np.random.default_rng(2)
    omega = (rng.random((12, 8, 16)) > 0.7).astype(float)
    phi = oracle.pfs(omega, 2, 0.0, threshold=0.0)
    blocks = omega.reshape(6, 2, 4, 2, 8, 2).mean(axis=(1, 3, 5))
    assert np.allclose(phi, blocks, rtol=0, atol=1e-13)
    cut = oracle.pfs(omega, 2, 1.0, threshold=0.05)
    ref = oracle.pfs(omega, 2, 1.0, threshold=0.0)
    assert np.array_equal(cut, np.where(ref < 0.05, 0.0, ref))


def test_filtered_indicator_stays_in_the_unit_interval():
    """the Green's function of 1 - c lap is positive and sums to one"""
    omega, _ = ri.octet(16, 0.2)
    omega = (omega > 0.5).astype(float)
    phi = oracle.pfs(omega, 2, 1.0, threshold=0.0)
    assert phi.min() >= -1e-12 and phi.max() <= 1 + 1e-12
