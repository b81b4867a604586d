"""Pins of the oracle's J2 plasticity and Newton extension (section 2.1.1,
section 5): the radial return against its defining conditions, the
consistent tangent against finite differences of the return map, uniaxial
loading of a homogeneous cell against the elastoplastic closed forms derived
by hand, an elastic increment against the pinned linear mixed-control solve,
and a plastic increment on an octet meeting its constraints."""
import numpy as np
import pytest

import oracle
import rve_inputs as ri

E_M, NU_M, SY = 110e9, 0.3, 70e6
M = np.array([1.0, 1, 1, 0, 0, 0])


def dev_norm(s):
    return np.linalg.norm(s - s[:3].mean() * M)


@pytest.mark.parametrize("H", [0.0, E_M / 50])
def test_return_map_meets_yield_condition_and_flow_rule(H):
    rng = np.random.default_rng(0)
    for k in range(20):
        eps = rng.standard_normal(6) * 3e-3
        epsp = rng.standard_normal(6) * 1e-4
        epsp -= epsp[:3].mean() * M                  # plastic strain is deviatoric
        a0 = abs(rng.standard_normal()) * 1e-3
        phi = 0.3 + 0.7 * rng.random()
        sig, Ct, epn, a1 = oracle.j2_point(E_M, NU_M, SY, H, phi, eps, epsp, a0)
        s = sig / phi
        radius = np.sqrt(2 / 3) * (SY + H * a1)
        assert dev_norm(s) <= radius * (1 + 1e-12)
        dp = epn - epsp
        if np.linalg.norm(dp) > 0:
            assert dev_norm(s) == pytest.approx(radius, rel=1e-12)          # on the yield surface
            assert abs(dp[:3].sum()) <= 1e-15                                # isochoric flow
            sd = s - s[:3].mean() * M
            assert np.allclose(dp / np.linalg.norm(dp), sd / np.linalg.norm(sd), atol=1e-12)   # normal to it
            assert a1 - a0 == pytest.approx(np.sqrt(2 / 3) * np.linalg.norm(dp), rel=1e-12)


@pytest.mark.parametrize("H", [0.0, E_M / 50])
def test_consistent_tangent_is_the_derivative_of_the_return_map(H):
    rng = np.random.default_rng(1)
    for k in range(10):
        eps = rng.standard_normal(6) * 2e-3
        epsp = np.zeros(6)
        sig, Ct, _, _ = oracle.j2_point(E_M, NU_M, SY, H, 0.8, eps, epsp, 0.0)
        h = 1e-9
        fd = np.zeros((6, 6))
        for j in range(6):
            d = np.zeros(6)
            d[j] = h
            fd[:, j] = (oracle.j2_point(E_M, NU_M, SY, H, 0.8, eps + d, epsp, 0.0)[0] -
                        oracle.j2_point(E_M, NU_M, SY, H, 0.8, eps - d, epsp, 0.0)[0]) / (2 * h)
        assert np.allclose(Ct, fd, rtol=0, atol=1e-5 * np.max(np.abs(Ct)))


@pytest.mark.parametrize("H", [0.0, E_M / 20])
def test_homogeneous_uniaxial_loading_follows_the_closed_form(H):
    """e11 prescribed, other components stress-free: below yield s = E e;
    beyond, with s = sy + H e_p and e = s / E + e_p (uniaxial J2 with the
    sqrt(2/3) hardening convention), |s| = (sy + H |e|) / (1 + H / E)."""
    c = 0.6
    cell = oracle.J2Cell(np.full((4, 4, 4), c), E_M, NU_M, SY, H)
    for k in range(1, 9):
        e = -2e-4 * k
        out = cell.increment(0b111110, [e, 0, 0, 0, 0, 0], np.zeros(6))
        assert out["accepted"]
        ey = SY / E_M
        s = E_M * abs(e) if abs(e) <= ey else (SY + H * abs(e)) / (1 + H / E_M)
        assert out["sigma_mean"][0] == pytest.approx(-c * s, rel=1e-9)
        assert np.allclose(out["sigma_mean"][1:], 0, atol=1e-9 * c * s)


def test_elastic_increment_equals_the_linear_mixed_solve():
    phi, _ = ri.octet(12, 0.2)
    cell = oracle.J2Cell(phi, E_M, NU_M, 1e12, 0.0)          # never yields
    Ebar = np.array([-2e-4, 0, 0, 0, 0, 0])
    out = cell.increment(0b111110, Ebar, np.zeros(6), tol_lin=1e-10)
    ref = oracle.solve_mixed(phi, E_M, NU_M, 1, 0b111110, Ebar, np.zeros(6), tol=1e-12, max_it=5000)
    assert out["accepted"]
    assert np.allclose(out["sigma_mean"], ref["sigma_mean"], rtol=0, atol=1e-7 * abs(ref["sigma_mean"][0]))
    assert np.allclose(out["eps_mean"], ref["eps_mean"], rtol=0, atol=1e-7 * abs(ref["eps_mean"][0]))


def test_plastic_increments_on_an_octet_meet_their_constraints():
    """With a small hardening the damped Newton method accepts each
    increment; the lateral mean stresses stay zero, the prescribed e11 is
    met, every solid voxel lies inside its yield surface, and the struts
    have yielded."""
    phi, _ = ri.octet(12, 0.2)
    cell = oracle.J2Cell(phi, E_M, NU_M, SY, E_M / 100)
    for k in range(1, 4):
        e = -5e-3 * k
        out = cell.increment(0b111110, [e, 0, 0, 0, 0, 0], np.zeros(6))
        assert out["accepted"]
        s11 = abs(out["sigma_mean"][0])
        assert np.all(np.abs(out["sigma_mean"][1:]) <= 1e-4 * s11)
        assert out["eps_mean"][0] == pytest.approx(e, rel=1e-10)
    assert (cell.alpha[phi > 0.5] > 0).mean() > 0.5


@pytest.mark.parametrize("H", [0.0, E_M / 50])
def test_consistent_tangent_eigen_structure(H):
    """For associative J2 with isotropic hardening the consistent tangent of
    the radial return is symmetric; in a plastic state it maps the flow
    direction n (the unit deviatoric stress) to phi 2 mu H / (3 mu + H) n,
    the hardening stiffness of the continuum law (zero for perfect
    plasticity), and the volumetric direction m to phi 3 kappa m (J2 flow is
    isochoric); in an elastic state it is phi C_m."""
    lam = E_M * NU_M / ((1 + NU_M) * (1 - 2 * NU_M))
    mu = E_M / (2 * (1 + NU_M))
    kappa = lam + 2 * mu / 3
    rng = np.random.default_rng(7)
    seen = {True: 0, False: 0}
    for k in range(40):
        scale = 3e-3 if k % 2 else 2e-4                # plastic and elastic states
        eps = rng.standard_normal(6) * scale
        epsp = np.zeros(6)
        phi = 0.3 + 0.7 * rng.random()
        sig, Ct, _, a1 = oracle.j2_point(E_M, NU_M, SY, H, phi, eps, epsp, 0.0)
        assert np.abs(Ct - Ct.T).max() <= 1e-14 * np.abs(Ct).max()
        assert np.allclose(Ct @ M, phi * 3 * kappa * M, rtol=0, atol=1e-12 * phi * kappa)
        plastic = a1 > 0
        seen[plastic] += 1
        if plastic:
            s = sig / phi
            dev = s - s[:3].mean() * M
            n = dev / np.linalg.norm(dev)
            assert np.allclose(Ct @ n, phi * 2 * mu * H / (3 * mu + H) * n, rtol=0, atol=1e-12 * phi * mu)
        else:
            Cm = np.zeros((6, 6))
            Cm[:3, :3] = lam
            Cm += 2 * mu * np.eye(6)
            assert np.allclose(Ct, phi * Cm, rtol=0, atol=1e-12 * phi * mu)
    assert seen[True] > 5 and seen[False] > 5


def test_section5_compression_curve_with_the_paper_material():
    """Section 5's test on a dense octet (rho = 0.3, 12^3): PA12 (E = 1.7
    GPa, nu = 0.4), perfect plasticity at 70 MPa, compression to -10 % in 20
    increments with stress-free lateral faces.  Every increment is accepted;
    the first ones are elastic, so the stress is proportional to the strain
    with the slope of the pinned linear mixed solve; past yield the curve
    flattens (a plastic regime with a small apparent hardening rate)."""
    E, nu, sy = 1.7e9, 0.4, 70e6
    phi, _ = ri.octet(12, 0.3)
    phi = phi.astype(np.float64)
    cell = oracle.J2Cell(phi, E, nu, sy, 0.0)
    s11 = []
    for k in range(1, 21):
        out = cell.increment(0b111110, [-0.005 * k, 0, 0, 0, 0, 0], np.zeros(6))
        assert out["accepted"]
        assert np.all(np.abs(out["sigma_mean"][1:]) <= 1e-4 * abs(out["sigma_mean"][0]))
        s11.append(out["sigma_mean"][0])
    lin = oracle.solve_mixed(phi, E, nu, 1, 0b111110, [-0.005, 0, 0, 0, 0, 0], np.zeros(6), tol=1e-10)
    assert s11[0] == pytest.approx(lin["sigma_mean"][0], rel=1e-5)
    assert s11[1] == pytest.approx(2 * s11[0], rel=1e-5)
    assert all(b < a for a, b in zip(s11, s11[1:]))                  # monotone in compression
    elastic_slope = s11[0] / -0.005
    final_slope = (s11[-1] - s11[-2]) / -0.005
    assert 0 < final_slope < 0.3 * elastic_slope
    assert (cell.alpha[phi > 0.5] > 0).any()
