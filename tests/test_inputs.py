"""Input generators: geometry only (none of the method's arithmetic)."""
import numpy as np

import rve_inputs as ri


def test_octet_density_and_symmetry():
    phi, r = ri.octet(24, 0.15)
    assert abs(phi.mean() - 0.15) < 2e-3
    assert 0 < r < 0.2
    # cubic symmetry of the FCC truss: axis permutations map the cell onto itself
    assert np.allclose(phi, phi.transpose(1, 0, 2), atol=1e-6)
    assert np.allclose(phi, phi.transpose(2, 1, 0), atol=1e-6)


def test_grf_statistics():
    f = ri.gaussian_random_field(64, seed=3, corr_len=3.0, std=1.0)
    assert abs(f.mean()) < 1e-5 and abs(f.std() - 1.0) < 1e-4
    # correlation at lag 3 voxels: exp(-9 / (2 * 9)) = 0.61 for the Gaussian covariance
    c3 = np.mean(f * np.roll(f, 3, axis=0))
    assert 0.5 < c3 < 0.72


def test_as_printed_small():
    phi, r = ri.as_printed(64, cells=2, rho=0.12, seed=5)
    assert 0.10 < phi.mean() < 0.125          # 12 % before pores, about 1 % of it carved
    assert phi.min() >= 0 and phi.max() <= 1
    rough, _ = ri.octet(64, 0.12, cells=2)
    assert np.abs(phi - rough).mean() > 1e-3  # the surface moved


def test_band_voxelizer_matches_full_sampling():
    """The radius search classifies voxels far from the surface without
    sub-sampling them; with the random-field perturbation that shortcut must
    still give exactly what sub-sampling every voxel gives."""
    n = 32
    grf = ri.gaussian_random_field(n, seed=2) * (2.0 / n)
    phi, r = ri.octet(n, 0.12, cells=2, dist_perturb=grf)
    full = ri.octet_at_radius(n, r, cells=2, dist_perturb=grf)
    assert np.array_equal(phi, full)
    assert abs(phi.mean() - 0.12) < 1.0 / (64 * n ** 3) + 1e-7
    plain, r0 = ri.octet(n, 0.12, cells=2)
    assert np.array_equal(plain, ri.octet_at_radius(n, r0, cells=2))


def test_octet_family_matches_the_voxelizer():
    fam = ri.OctetFamily(24)
    for rho in (0.05, 0.15, 0.3):
        phi, r = ri.octet(24, rho)
        assert fam.radius(rho) == r
        assert np.array_equal(fam.phi(rho), phi)


def test_va_phase_is_the_volume_fraction_at_a_planar_surface():
    """Material x < a: the voxel [i, i+1) holds the fraction clip(a - i, 0, 1)
    of material, and the Voigt analytic map reproduces it exactly."""
    for a in (3.0, 3.2, 3.5, 3.87, 4.0):
        centres = np.arange(8) + 0.5
        phi = ri.va_phase(a - centres, 1.0)
        expect = np.clip(a - np.arange(8), 0.0, 1.0)
        assert np.allclose(phi, expect, rtol=0, atol=1e-15)


def test_octet_va_approaches_the_subsampled_voigt_map():
    """The paper finds the Voigt analytic map almost identical to the fine-
    grid Voigt rule (section 3.3): the mean density of the two agrees to 0.5 %
    at 64^3 (it is 1.5 % at 32^3) and the voxel-wise difference shrinks with
    the grid."""
    diffs = []
    for n in (32, 64):
        va, r = ri.octet_va(n, 0.15)
        vfg = ri.octet_at_radius(n, r, sub=8)
        assert va.min() >= 0.0 and va.max() <= 1.0
        diffs.append(float(np.abs(va - vfg).mean()))
        if n == 64:
            assert abs(va.mean() - vfg.mean()) <= 5e-3 * vfg.mean()
    assert diffs[1] < diffs[0]
