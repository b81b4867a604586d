"""GPU parity of the elastoplastic Newton extension (hom_j2_*; section 2.1.1,
the J2 lattice material of section 5) against the FP64 oracle and against
closed forms.

Both sides run the same damped Newton method in FP64 (the GPU's FP32-field
mode differs only in solving the Newton systems in FP32).  Where the cell has
no void (the octet with its empty voxels at 5 % of the material) the
linearised systems are definite, the Newton iterates converge to
tol_lin = 1e-9, tol_newton = 1e-7, and a perturbation of the inputs at
round-off size moves the result by about 1e-10: there mean stresses and
strains must agree to 1e-7 (relative to the largest), the strain, plastic
strain and hardening fields to 1e-6 in L2.  With void the Newton path is
chaotic (a round-off perturbation of E changes the fields of a three-
increment path at the default tolerances by up to 20 %), so the void octet
is compared one Newton step per increment (max_newton = 1), where the same
perturbation moves the fields by about 1.6e-5 and the means by 3e-6: 2e-4
(fields on phi > 0; the void admits strain fields that carry no stress) and
2e-5 (means).  Full increments on the void octet are checked against their
constraints.  Homogeneous and elastic cases follow closed forms or the
linear mixed solve."""
import numpy as np
import pytest

import oracle
import rve_inputs as ri

pytestmark = pytest.mark.gpu

E_M, NU_M, SY = 110e9, 0.3, 70e6
TL, TN = 1e-9, 1e-7


@pytest.fixture(scope="module")
def hom():
    import torch
    assert torch.cuda.is_available()
    from paper_2110_00733_gb300 import build, hom as h
    build.build()
    h.load_library()
    return h


PRECS = {"fp64": 1, "fp32": 0}   # HOM_PREC_FP64, HOM_PREC_FP32_FIELDS


def make(hom, phi, prec=None):
    p = hom.HOM_PREC_FP64 if prec is None else prec
    return hom.hom_create(phi.shape, np.ascontiguousarray(phi, dtype=np.float64), hom.HOM_INPUT_FRACTION_F64,
                          E_M, NU_M, precision=p)


def rel_l2(a, b, where):
    den = np.linalg.norm(b[..., where])
    return np.linalg.norm((a - b)[..., where]) / (den if den > 0 else 1.0)


LOADS = {
    # uniaxial stress in e11 (lateral means stress-free), compression into the plastic range
    "uniaxial": (0b111110, [np.array([-2e-3 * k, 0, 0, 0, 0, 0]) for k in (1, 2, 3)]),
    # strain-controlled shear with a little volumetric strain, all six means prescribed
    "shear": (0, [np.array([1e-4, 0, 0, 0, 0, 1.5e-3]) * k for k in (1, 2)]),
}


def compare(hom, ctx, cell, ref, got, where, mtol, ftol):
    assert np.max(np.abs(got["sigma_mean"] - ref["sigma_mean"])) <= mtol * np.max(np.abs(ref["sigma_mean"]))
    assert np.max(np.abs(got["eps_mean"] - ref["eps_mean"])) <= mtol * np.max(np.abs(ref["eps_mean"]))
    eps, epsp, alpha = hom.hom_j2_state(ctx)
    assert rel_l2(eps, oracle.mandel_to_tensor(cell.eps), where) <= ftol
    assert rel_l2(epsp, oracle.mandel_to_tensor(cell.epsp), where) <= ftol
    assert rel_l2(alpha, cell.alpha, where) <= ftol
    return alpha


@pytest.mark.parametrize("H", [E_M / 20, E_M / 100])
@pytest.mark.parametrize("shape,load", [((16, 16, 16), "uniaxial"), ((12, 16, 10), "shear")])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_increments_match_oracle(hom, shape, load, H, prec):
    """FP32 fields solve the Newton systems in FP32 (to 1e-6; Newton to
    1e-5) while strains, history and residuals stay FP64: their accepted
    iterates are compared with the oracle's tight ones at 2e-5 (means) and
    1e-4 (fields)."""
    phi, _ = ri.octet(shape if len(set(shape)) > 1 else shape[0], 0.2)
    phi = 0.05 + 0.95 * phi.astype(np.float64)
    mask, path = LOADS[load]
    cell = oracle.J2Cell(phi, E_M, NU_M, SY, H)
    fp64 = prec == "fp64"
    tl, tn = (TL, TN) if fp64 else (1e-6, 1e-5)
    with make(hom, phi, PRECS[prec]) as ctx:
        hom.hom_j2_begin(ctx, SY, H)
        for Ebar in path:
            ref = cell.increment(mask, Ebar, np.zeros(6), tol_lin=TL, tol_newton=TN)
            rc, got = hom.hom_j2_increment(ctx, Ebar, np.zeros(6), mask, tol_lin=tl, tol_newton=tn)
            assert ref["accepted"] and rc == hom.HOM_OK and got["accepted"]
            if fp64:
                assert abs(got["newton"] - ref["newton"]) <= 1
            alpha = compare(hom, ctx, cell, ref, got, phi > 0, 1e-7 if fp64 else 2e-5, 1e-6 if fp64 else 1e-4)
        assert (alpha[phi > 0.5] > 0).mean() > 0.1      # the struts have yielded


def test_single_newton_steps_on_the_void_octet_match_oracle(hom):
    phi, _ = ri.octet(16, 0.2)
    phi = phi.astype(np.float64)
    H = E_M / 100
    cell = oracle.J2Cell(phi, E_M, NU_M, SY, H)
    with make(hom, phi) as ctx:
        hom.hom_j2_begin(ctx, SY, H)
        for k in range(1, 4):
            Ebar = np.array([-1.5e-3 * k, 0, 0, 0, 0, 0])
            ref = cell.increment(0b111110, Ebar, np.zeros(6), max_newton=1)
            rc, got = hom.hom_j2_increment(ctx, Ebar, np.zeros(6), 0b111110, max_newton=1)
            assert rc == hom.HOM_NOT_CONVERGED and got["newton"] == 1
            assert got["residual"] == pytest.approx(ref["residual"], rel=1e-3)
            compare(hom, ctx, cell, ref, got, phi > 0, 2e-5, 2e-4)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_plastic_increments_on_the_void_octet_meet_their_constraints(hom, prec):
    """full increments with the default tolerances: accepted, lateral mean
    stresses zero, the prescribed e11 met, every voxel inside its yield
    surface, the struts yielded"""
    phi, _ = ri.octet(12, 0.2)
    phi = phi.astype(np.float64)
    H = E_M / 100
    with make(hom, phi, PRECS[prec]) as ctx:
        hom.hom_j2_begin(ctx, SY, H)
        for k in range(1, 4):
            e = -5e-3 * k
            rc, out = hom.hom_j2_increment(ctx, [e, 0, 0, 0, 0, 0], np.zeros(6), 0b111110, max_newton=60)
            assert rc == hom.HOM_OK
            s11 = abs(out["sigma_mean"][0])
            assert np.all(np.abs(out["sigma_mean"][1:]) <= 1e-4 * s11)
            assert out["eps_mean"][0] == pytest.approx(e, rel=1e-10)
        eps, epsp, alpha = hom.hom_j2_state(ctx)
        assert (alpha[phi > 0.5] > 0).mean() > 0.5
        # stress of the history: phi times the return of the elastic strain, on the yield surface or inside
        r2 = np.sqrt(2.0)
        ee = oracle.tensor_to_mandel(eps - epsp)
        lam, mu = E_M * NU_M / ((1 + NU_M) * (1 - 2 * NU_M)), E_M / (2 * (1 + NU_M))
        s = 2 * mu * ee
        s[:3] += lam * ee[:3].sum(axis=0)
        dev = s.copy()
        dev[:3] -= s[:3].mean(axis=0)
        radius = np.sqrt(2 / 3) * (SY + H * alpha)
        assert np.all(np.sqrt((dev ** 2).sum(axis=0)) <= radius * (1 + 1e-8) + 1e-12 * r2)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("H", [0.0, E_M / 20])
def test_homogeneous_uniaxial_loading_follows_the_closed_form(hom, H, prec):
    """e11 prescribed, lateral means stress-free: below yield s = E e, beyond
    |s| = (sy + H |e|) / (1 + H / E) (uniaxial J2, sqrt(2/3) hardening
    convention), times phi; unloading is elastic."""
    c = 0.6
    rel = 1e-9 if prec == "fp64" else 1e-6
    with make(hom, np.full((8, 8, 8), c), PRECS[prec]) as ctx:
        hom.hom_j2_begin(ctx, SY, H)
        ey = SY / E_M
        for k in range(1, 9):
            e = -2e-4 * k
            rc, out = hom.hom_j2_increment(ctx, [e, 0, 0, 0, 0, 0], np.zeros(6), 0b111110)
            assert rc == hom.HOM_OK
            s = E_M * abs(e) if abs(e) <= ey else (SY + H * abs(e)) / (1 + H / E_M)
            assert out["sigma_mean"][0] == pytest.approx(-c * s, rel=rel)
            assert np.allclose(out["sigma_mean"][1:], 0, atol=rel * c * s)
        # elastic unloading by de = 1e-4 from the last state
        s_last = out["sigma_mean"][0]
        rc, out = hom.hom_j2_increment(ctx, [e + 1e-4, 0, 0, 0, 0, 0], np.zeros(6), 0b111110)
        assert rc == hom.HOM_OK
        assert out["sigma_mean"][0] == pytest.approx(s_last + c * E_M * 1e-4, rel=rel)


def test_elastic_increment_equals_the_mixed_solve(hom):
    """with a yield stress never reached one Newton step solves the linear
    mixed problem: means equal those of hom_solve_mixed"""
    phi, _ = ri.octet(16, 0.2)
    phi = 0.05 + 0.95 * phi.astype(np.float64)
    Ebar = np.array([-2e-4, 0, 0, 0, 0, 0])
    with make(hom, phi) as ctx:
        rc, lin = hom.hom_solve_mixed(ctx, Ebar[None], np.zeros((1, 6)), 0b111110, tol=1e-11, max_it=6000)
        assert rc == hom.HOM_OK
        hom.hom_j2_begin(ctx, 1e12, 0.0)
        rc, out = hom.hom_j2_increment(ctx, Ebar, np.zeros(6), 0b111110, tol_lin=1e-11, max_lin=6000)
        assert rc == hom.HOM_OK and out["newton"] <= 2
        sm, em = lin[0]["sigma_mean"], lin[0]["eps_mean"]
        assert np.max(np.abs(out["sigma_mean"] - sm)) <= 1e-7 * abs(sm[0])
        assert np.max(np.abs(out["eps_mean"] - em)) <= 1e-7 * abs(em[0])


def test_linear_solves_after_a_plastic_increment_are_unchanged(hom):
    """the solve graph captured with the tangent operator is replaced when
    hom_solve runs next: its result equals that of a fresh context"""
    phi, _ = ri.octet(16, 0.2)
    phi = phi.astype(np.float64)
    E = np.eye(6)[[0, 5]] * 1e-3
    with make(hom, phi) as fresh:
        _, ref = hom.hom_solve(fresh, E, tol=1e-10, max_it=4000)
    with make(hom, phi) as ctx:
        hom.hom_j2_begin(ctx, SY, E_M / 100)
        rc, _ = hom.hom_j2_increment(ctx, [-3e-3, 0, 0, 0, 0, 0], np.zeros(6), 0b111110, max_newton=3)
        assert rc in (hom.HOM_OK, hom.HOM_NOT_CONVERGED)
        rc, got = hom.hom_solve(ctx, E, tol=1e-10, max_it=4000)
        assert rc == hom.HOM_OK
        for g, r in zip(got, ref):
            assert np.allclose(g["sigma_mean"], r["sigma_mean"], rtol=1e-12, atol=1e-9)
        # and a later increment resumes from the kept history
        rc, out = hom.hom_j2_increment(ctx, [-4e-3, 0, 0, 0, 0, 0], np.zeros(6), 0b111110, max_newton=3)
        assert rc in (hom.HOM_OK, hom.HOM_NOT_CONVERGED)
        assert out["eps_mean"][0] == pytest.approx(-4e-3, rel=1e-12)


def test_j2_rejections(hom):
    phi = np.full((8, 8, 8), 0.5)
    with hom.hom_create(phi.shape, phi, hom.HOM_INPUT_FRACTION_F64, E_M, NU_M,
                        solver=hom.HOM_SOLVER_MODBFFT_CG) as ctx:
        with pytest.raises(hom.HomError) as e:
            hom.hom_j2_begin(ctx, SY, 0.0)
        assert e.value.code == hom.HOM_EINVAL
    with make(hom, phi) as ctx:
        with pytest.raises(hom.HomError) as e:
            hom.hom_j2_increment(ctx, np.zeros(6), np.zeros(6), 0)
        assert e.value.code == hom.HOM_EINVAL
        with pytest.raises(hom.HomError) as e:
            hom.hom_j2_begin(ctx, -1.0, 0.0)
        assert e.value.code == hom.HOM_EINVAL
        hom.hom_j2_begin(ctx, SY, 0.0)
        with pytest.raises(hom.HomError) as e:
            hom.hom_j2_increment(ctx, np.zeros(6), np.zeros(6), 64)
        assert e.value.code == hom.HOM_EINVAL
        # a zero increment from the virgin state needs no Newton step
        rc, out = hom.hom_j2_increment(ctx, np.zeros(6), np.zeros(6), 0)
        assert rc == hom.HOM_OK and out["newton"] == 0
        hom.hom_j2_end(ctx)
        with pytest.raises(hom.HomError) as e:
            hom.hom_j2_state(ctx)
        assert e.value.code == hom.HOM_EINVAL
