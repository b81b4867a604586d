"""Pins of the oracle's mixed macroscopic control (eq. galop: the projector at
xi = 0 is the symmetric identity on the stress-controlled components KL and
zero on the strain-controlled kl; eq. gallin: the right-hand side carries
C : Ebar - Sbar).  The solution's mean then holds the unknown mean strain of
the KL components.

The pins do not go through the oracle's own stiffness routine: the
homogeneous cell is checked against the isotropic compliance written out,
and the heterogeneous cell against the compliance obtained by inverting the
strain-controlled effective stiffness (six independent solves)."""
import numpy as np
import pytest

import oracle
import rve_inputs as ri

E_M, NU_M = 110e9, 0.3
ALL = 0b111111          # every Mandel component stress-controlled
LATERAL = 0b111110      # e11 prescribed, the other five stress-free


def voigt_strain(eps_t):
    """tensor strain components -> Voigt (engineering shears)"""
    e = np.array(eps_t, dtype=np.float64)
    e[3:] *= 2.0
    return e


@pytest.mark.parametrize("deriv", [0, 1])
def test_homogeneous_cell_follows_isotropic_compliance(deriv):
    """phi = c: the stress is uniform and the strain is the isotropic
    compliance of c C_m applied to it, e11 = s / (c E), e22 = e33 = -nu s /
    (c E), e23 = t / (2 c mu)."""
    c = 0.37
    phi = np.full((6, 5, 4), c)
    s, t = 2.0e6, 0.7e6
    Sbar = np.array([s, 0, 0, t, 0, 0])
    out = oracle.solve_mixed(phi, E_M, NU_M, deriv, ALL, np.zeros(6), Sbar, tol=1e-12)
    mu = E_M / (2 * (1 + NU_M))
    expect = np.array([s / (c * E_M), -NU_M * s / (c * E_M), -NU_M * s / (c * E_M), t / (2 * c * mu), 0, 0])
    assert np.allclose(out["eps_mean"], expect, rtol=0, atol=1e-12 * abs(expect[0]))
    assert np.allclose(out["sigma_mean"], Sbar, rtol=0, atol=1e-9 * s)
    # the solution is the uniform strain (Mandel field, constant per component)
    field = out["eps_tilde"].reshape(6, -1)
    assert np.allclose(field, oracle.tensor_to_mandel(expect)[:, None], rtol=0, atol=1e-12 * abs(expect[0]))


def test_homogeneous_uniaxial_strain_with_free_lateral_faces():
    """e11 prescribed, the other five components stress-free: uniaxial
    stress, s11 = c E e11 and e22 = e33 = -nu e11."""
    c = 0.8
    phi = np.full((4, 6, 5), c)
    e = 1e-3
    out = oracle.solve_mixed(phi, E_M, NU_M, 1, LATERAL, np.array([e, 0, 0, 0, 0, 0]), np.zeros(6), tol=1e-12)
    assert out["sigma_mean"][0] == pytest.approx(c * E_M * e, rel=1e-10)
    assert np.allclose(out["sigma_mean"][1:], 0, atol=1e-10 * c * E_M * e)
    assert np.allclose(out["eps_mean"], [e, -NU_M * e, -NU_M * e, 0, 0, 0], rtol=0, atol=1e-12 * e)


def test_no_stress_control_ignores_sbar_and_equals_strain_control():
    phi, _ = ri.octet(8, 0.2)
    Ebar = np.array([1e-3, 0, 0, 0, 2e-4, 0])
    a = oracle.solve(phi, E_M, NU_M, 1, Ebar, tol=1e-10)
    b = oracle.solve_mixed(phi, E_M, NU_M, 1, 0, Ebar, np.array([5e6, 1, 2, 3, 4, 5.0]), tol=1e-10)
    assert np.array_equal(a["eps_tilde"], b["eps_tilde"])
    assert np.array_equal(a["sigma_mean"], b["sigma_mean"])
    assert np.allclose(b["eps_mean"], Ebar, rtol=0, atol=1e-16)


@pytest.fixture(scope="module")
def octet_compliance():
    """Compliance of a 12^3 octet from the six strain-controlled solves."""
    phi, _ = ri.octet(12, 0.15)
    C, _ = oracle.effective_stiffness(phi, E_M, NU_M, 1, tol=1e-11, max_it=4000)
    return phi, np.linalg.inv(C)


def test_uniaxial_stress_strain_is_the_compliance_column(octet_compliance):
    """All six components stress-controlled, Sbar = s e1 (x) e1: the mean
    strain is S s e1 in Voigt form, the first column of the inverse of the
    strain-controlled C_eff; the mean stress equals Sbar."""
    phi, S = octet_compliance
    s = 1.0e6
    Sbar = np.array([s, 0, 0, 0, 0, 0])
    out = oracle.solve_mixed(phi, E_M, NU_M, 1, ALL, np.zeros(6), Sbar, tol=1e-11, max_it=4000)
    assert out["true_residual"] < 1e-9
    ev = voigt_strain(out["eps_mean"])
    assert np.allclose(ev, S[:, 0] * s, rtol=0, atol=1e-7 * abs(S[0, 0] * s))
    assert np.allclose(out["sigma_mean"], Sbar, rtol=0, atol=1e-9 * s)
    # Young's modulus and Poisson ratio of the cell from this one solve
    E_eff, nu_eff = s / ev[0], -ev[1] / ev[0]
    assert E_eff == pytest.approx(1.0 / S[0, 0], rel=1e-7)
    assert nu_eff == pytest.approx(-S[1, 0] / S[0, 0], rel=1e-6)


def test_prescribed_axial_strain_with_free_faces_gives_E_and_nu(octet_compliance):
    """e11 prescribed, the other components stress-free: s11 = e11 / S11 and
    the lateral strains are S21 s11, S31 s11."""
    phi, S = octet_compliance
    e = 1e-3
    out = oracle.solve_mixed(phi, E_M, NU_M, 1, LATERAL, np.array([e, 0, 0, 0, 0, 0]), np.zeros(6),
                             tol=1e-11, max_it=4000)
    s11 = e / S[0, 0]
    assert out["sigma_mean"][0] == pytest.approx(s11, rel=1e-7)
    assert np.allclose(out["sigma_mean"][1:], 0, atol=1e-9 * abs(s11))
    assert out["eps_mean"][0] == pytest.approx(e, rel=1e-14)
    assert np.allclose(voigt_strain(out["eps_mean"])[1:], S[1:, 0] * s11, rtol=0, atol=1e-7 * e)


def test_mixed_load_meets_both_constraints(octet_compliance):
    """A general mixed load: prescribed strains where the mask is clear,
    prescribed stresses where it is set, and the mean strain and stress of
    the solution are tied by the compliance."""
    phi, S = octet_compliance
    mask = 0b101010                      # s22, s23, s12 prescribed; e11, e33, e13 prescribed
    Ebar = np.array([8e-4, 0, -3e-4, 0, 2e-4, 0])
    Sbar = np.array([0, 4e6, 0, -1e6, 0, 2.5e6])
    out = oracle.solve_mixed(phi, E_M, NU_M, 1, mask, Ebar, Sbar, tol=1e-11, max_it=4000)
    for c in range(6):
        if (mask >> c) & 1:
            assert out["sigma_mean"][c] == pytest.approx(Sbar[c], rel=1e-8, abs=1e-3)
        else:
            assert out["eps_mean"][c] == pytest.approx(Ebar[c], rel=1e-12, abs=1e-18)
    ev = voigt_strain(out["eps_mean"])
    assert np.allclose(ev, S @ out["sigma_mean"], rtol=0, atol=1e-7 * np.max(np.abs(ev)))
