"""GPU parity of conjugate gradients on the Galerkin system
(HOM_SOLVER_GALERKIN_CG; section 2.1) against the oracle's CG, and the
behaviour around section 2.1: CG converges where the cell has no void, and
with the rotated scheme on a lattice with void as well.

Tolerances as for MINRES: FP64 fields solve to 1e-8 and agree with the
oracle (1e-11) in mean stress to 1e-6 relative and in fields to 1e-4 (L2,
strains on solid voxels); FP32 fields (refinement sweeps) to 1e-5 and
1e-4."""
import numpy as np
import pytest

import oracle
import rve_inputs as ri

pytestmark = pytest.mark.gpu

E_M, NU_M = 110e9, 0.3


@pytest.fixture(scope="module")
def hom():
    import torch
    assert torch.cuda.is_available()
    from paper_2110_00733_gb300 import build, hom as h
    build.build()
    h.load_library()
    return h


def make(hom, phi, prec, deriv, solver):
    p = hom.HOM_PREC_FP32_FIELDS if prec == "fp32" else hom.HOM_PREC_FP64
    return hom.hom_create(phi.shape, np.ascontiguousarray(phi, dtype=np.float64), hom.HOM_INPUT_FRACTION_F64,
                          E_M, NU_M, derivative=deriv, precision=p, solver=solver)


def check_fields(hom, ctx, phi, ref, Ebar, tol):
    strain, stress = hom.hom_fields(ctx, 0)
    eps_ref = oracle.mandel_to_tensor(ref["eps_tilde"]) + Ebar[:, None, None, None]
    solid = phi > 0
    assert np.linalg.norm((strain - eps_ref)[:, solid]) <= tol * np.linalg.norm(eps_ref[:, solid])
    Cm = oracle.stiffness_mandel(E_M, NU_M)
    sig_ref = oracle.mandel_to_tensor(np.einsum("ij,j...->i...", Cm, oracle.tensor_to_mandel(eps_ref)) * phi)
    assert np.linalg.norm(stress - sig_ref) <= tol * np.linalg.norm(sig_ref)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("deriv", [0, 1])
def test_cg_matches_oracle_cg_without_void(hom, prec, deriv):
    phi, _ = ri.octet(16, 0.2)
    phi = 0.05 + 0.95 * phi.astype(np.float64)
    Ebar = np.array([1e-3, -2e-4, 0, 3e-4, 0, 0])
    ref = oracle.solve_mixed(phi, E_M, NU_M, deriv, 0, Ebar, np.zeros(6), tol=1e-11, max_it=3000, method="cg")
    with make(hom, phi, prec, deriv, hom.HOM_SOLVER_GALERKIN_CG) as ctx:
        rc, info = hom.hom_solve(ctx, Ebar[None], tol=1e-8, max_it=3000)
        assert rc == hom.HOM_OK
        assert info[0]["true_residual"] <= 1e-8
        rel = 1e-5 if prec == "fp32" else 1e-6
        sm = ref["sigma_mean"]
        assert np.max(np.abs(info[0]["sigma_mean"] - sm)) <= rel * np.max(np.abs(sm))
        check_fields(hom, ctx, phi, ref, Ebar, 1e-4)
        if prec == "fp64":
            # the same recurrence: the oracle at 1e-8 stops within an iteration of the GPU
            r8 = oracle.solve_mixed(phi, E_M, NU_M, deriv, 0, Ebar, np.zeros(6), tol=1e-8, max_it=3000,
                                    method="cg")
            assert abs(info[0]["iterations"] - r8["iterations"]) <= 1


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_cg_with_rotated_scheme_converges_on_lattice_with_void(hom, prec):
    """Rotated frequencies: CG reaches the MINRES solution on the octet with
    empty voxels (stresses and strains on the solid)."""
    phi, _ = ri.octet(16, 0.2)
    phi = phi.astype(np.float64)
    Ebar = np.array([1e-3, 0, 0, 0, 0, 0])
    ref = oracle.solve_mixed(phi, E_M, NU_M, 1, 0, Ebar, np.zeros(6), tol=1e-11, max_it=5000)
    with make(hom, phi, prec, 1, hom.HOM_SOLVER_GALERKIN_CG) as ctx:
        rc, info = hom.hom_solve(ctx, Ebar[None], tol=1e-8, max_it=5000)
        assert rc == hom.HOM_OK
        sm = ref["sigma_mean"]
        assert np.max(np.abs(info[0]["sigma_mean"] - sm)) <= 1e-5 * np.max(np.abs(sm))
        check_fields(hom, ctx, phi, ref, Ebar, 1e-4)


def test_continuous_scheme_with_void_leaves_the_stress_ill_determined(hom):
    """Continuous frequencies and empty voxels (section 2.1 motivates the
    rotated scheme and MINRES with this case).  MINRES converges; CG either
    stops unconverged or reaches the residual at a solution whose mean stress
    differs from MINRES's by a few tenths of a percent (0.24 % on this cell):
    modes that carry stress at almost no residual leave it undetermined to
    that level.  With the rotated scheme both agree to 1e-5 (test above)."""
    phi, _ = ri.octet(16, 0.2)
    Ebar = np.array([[1e-3, 0, 0, 0, 0, 0]])
    with make(hom, phi, "fp64", 0, hom.HOM_SOLVER_GALERKIN_MINRES) as ctx:
        rc, ref = hom.hom_solve(ctx, Ebar, tol=1e-6, max_it=4000)
        assert rc == hom.HOM_OK
    with make(hom, phi, "fp64", 0, hom.HOM_SOLVER_GALERKIN_CG) as ctx:
        rc, info = hom.hom_solve(ctx, Ebar, tol=1e-6, max_it=4000)
        if rc == hom.HOM_OK:
            assert info[0]["true_residual"] <= 1e-6
            sm = ref[0]["sigma_mean"]
            assert np.max(np.abs(info[0]["sigma_mean"] - sm)) <= 1e-2 * np.max(np.abs(sm))
        else:
            assert rc == hom.HOM_NOT_CONVERGED and info[0]["true_residual"] > 1e-6


def test_cg_under_mixed_control_matches_minres(hom):
    phi, _ = ri.octet(16, 0.2)
    phi = 0.05 + 0.95 * phi.astype(np.float64)
    Sbar = np.array([[1e6, 0, 0, 0, 0, 0]])
    out = []
    for solver in (hom.HOM_SOLVER_GALERKIN_MINRES, hom.HOM_SOLVER_GALERKIN_CG):
        with make(hom, phi, "fp64", 1, solver) as ctx:
            rc, info = hom.hom_solve_mixed(ctx, np.zeros((1, 6)), Sbar, 0b111111, tol=1e-9, max_it=3000)
            assert rc == hom.HOM_OK
            out.append(info[0])
    assert np.max(np.abs(out[0]["eps_mean"] - out[1]["eps_mean"])) <= 1e-7 * np.max(np.abs(out[0]["eps_mean"]))
