"""GPU parity: each step of the hot path through the C ABI against the FP64
oracle, element by element, on seeded inputs.

FP32 fields: max-abs error <= 2e-5 of the field's max |value| (FP32 FFT
round-off grows like u log2 V with u = 6e-8; 2e-5 leaves a margin of ~10 at
the sizes here).  FP64 fields: 1e-11."""
import numpy as np
import pytest

import oracle
import rve_inputs as ri
from gpu_util import FP32_TOL, FP64_TOL, half_spectrum, rel_maxerr

pytestmark = pytest.mark.gpu

E_M, NU_M = 110e9, 0.3
# several tiles and ragged tails on every axis; odd n3; mixed radices
SHAPES = [(8, 8, 8), (24, 20, 18), (12, 10, 9), (32, 32, 32), (30, 16, 40), (2, 6, 4), (5, 3, 50),
          (64, 64, 12), (128, 64, 10)]   # the last two run the TMA-staged n1/n2 passes in FP32
PRECS = ["fp32", "fp64"]


@pytest.fixture(scope="module")
def hom():
    import torch
    assert torch.cuda.is_available()
    from paper_2110_00733_gb300 import build, hom as h
    build.build()
    h.load_library()
    return h


def make(hom, phi, prec, deriv=1):
    p = hom.HOM_PREC_FP32_FIELDS if prec == "fp32" else hom.HOM_PREC_FP64
    return hom.hom_create(phi.shape, np.ascontiguousarray(phi, dtype=np.float64),
                          hom.HOM_INPUT_FRACTION_F64, E_M, NU_M, derivative=deriv, precision=p)


def tol(prec):
    return FP32_TOL if prec == "fp32" else FP64_TOL


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("shape", SHAPES)
def test_fft_forward_inverse(hom, shape, prec):
    phi = ri.random_phi(shape, seed=1)
    f = ri.random_field(shape, seed=sum(shape))
    with make(hom, phi, prec) as ctx:
        spec = hom.hom_fft_forward(ctx, f.astype(ctx.dtype))      # (n1, n2, h, 6)
        ref = np.stack([oracle.fft3d(f[c].astype(complex)) for c in range(6)])
        ref_h = np.moveaxis(half_spectrum(ref), 0, -1)
        assert rel_maxerr(spec, ref_h) <= tol(prec)
        back = hom.hom_fft_inverse(ctx, np.ascontiguousarray(ref_h.astype(spec.dtype)))
        assert rel_maxerr(back, f) <= tol(prec)


@pytest.mark.parametrize("deriv", [0, 1])
@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("shape", SHAPES)
def test_project_apply_rhs(hom, shape, prec, deriv):
    phi = ri.random_phi(shape, seed=2)
    f = ri.random_field(shape, seed=7)
    with make(hom, phi, prec, deriv) as ctx:
        got = hom.hom_project(ctx, f.astype(ctx.dtype))
        assert rel_maxerr(got, oracle.project(shape, deriv, f)) <= tol(prec)
        got = hom.hom_apply(ctx, f.astype(ctx.dtype))
        ref = oracle.apply(phi, 1.0, NU_M, deriv, f) * E_M   # library works in units of E
        assert rel_maxerr(got * E_M, ref) <= tol(prec)
        Eb = np.array([1e-3, -2e-4, 3e-4, 5e-4, -1e-4, 2e-4])
        got = hom.hom_rhs(ctx, Eb)
        ref = oracle.rhs(phi, 1.0, NU_M, deriv, Eb)
        assert rel_maxerr(got, ref) <= tol(prec)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("deriv", [1, 0])
def test_solve_octet_matches_oracle(hom, prec, deriv):
    """C_eff (6 unit strains) within 1e-4 relative; strain on solid voxels and
    stress everywhere within 1e-4 (L2), eq. (difff).

    Rotated frequencies: the octet cell with empty space (phi = 0).  The
    continuous scheme does not converge with zero-stiffness voxels (section
    2.1 says so and motivates the rotated scheme), so its case fills the
    void with a 5 % phase."""
    phi, _ = ri.octet(16, 0.2)
    phi = phi.astype(np.float64)
    if deriv == 0:
        phi = 0.05 + 0.95 * phi
    Cref, sols = oracle.effective_stiffness(phi, E_M, NU_M, deriv, tol=1e-11, max_it=5000)
    with make(hom, phi, prec, deriv) as ctx:
        rc, info = hom.hom_solve(ctx, np.eye(6), tol=1e-8, max_it=3000)
        assert rc == hom.HOM_OK, [i["status"] for i in info]
        C = hom.hom_effective_stiffness(ctx)
        assert np.max(np.abs(C - Cref)) <= 1e-4 * np.max(np.abs(Cref))
        for J in [0, 3]:
            strain, stress = hom.hom_fields(ctx, J)
            eps_ref = oracle.mandel_to_tensor(sols[J]["eps_tilde"]) + np.eye(6)[J][:, None, None, None]
            solid = phi > 0
            e_err = np.linalg.norm((strain - eps_ref)[:, solid]) / np.linalg.norm(eps_ref[:, solid])
            assert e_err <= 1e-4
            Cm = oracle.stiffness_mandel(E_M, NU_M)
            em = oracle.tensor_to_mandel(eps_ref)
            sig_ref = oracle.mandel_to_tensor(np.einsum("ij,j...->i...", Cm, em) * phi)
            s_err = np.linalg.norm(stress - sig_ref) / np.linalg.norm(sig_ref)
            assert s_err <= 1e-4
            assert info[J]["true_residual"] <= 1e-8


@pytest.mark.parametrize("prec", PRECS)
def test_laminate_closed_form_on_gpu(hom, prec):
    """Layered cell: exact laminate C_eff (the oracle's own pin), now on the GPU."""
    from test_oracle_solver import laminate_closed_form
    phi = ri.laminate((12, 6, 5), (4, 2, 6), (1.0, 0.2, 0.55), axis=0)
    with make(hom, phi, prec) as ctx:
        rc, info = hom.hom_solve(ctx, np.eye(6), tol=1e-9, max_it=500)
        assert rc == hom.HOM_OK
        for J in range(6):
            ref = laminate_closed_form([1.0, 0.2, 0.55], [4 / 12, 2 / 12, 6 / 12], np.eye(6)[J])
            assert np.allclose(info[J]["sigma_mean"], ref, rtol=1e-5, atol=1e-5 * E_M)


def test_homogeneous_cell_is_a_noop(hom):
    phi = np.full((8, 6, 10), 0.4)
    with make(hom, phi, "fp32") as ctx:
        rc, info = hom.hom_solve(ctx, np.eye(6), tol=1e-6, max_it=100)
        assert rc == hom.HOM_OK
        assert all(i["iterations"] == 0 for i in info)
        from test_oracle_solver import voigt_stiffness
        assert np.allclose(hom.hom_effective_stiffness(ctx), 0.4 * voigt_stiffness(E_M, NU_M), rtol=1e-6)


def test_errors_and_limits(hom):
    phi = ri.random_phi((8, 8, 8), seed=3)
    with pytest.raises(hom.HomError) as e:
        hom.hom_create((7, 8, 8), np.zeros((7, 8, 8)), hom.HOM_INPUT_FRACTION_F64, E_M, NU_M)
    assert e.value.code == hom.HOM_EUNSUPPORTED_GRID
    bad = phi.copy()
    bad[0, 0, 0] = np.nan
    with pytest.raises(hom.HomError) as e:
        hom.hom_create(bad.shape, bad, hom.HOM_INPUT_FRACTION_F64, E_M, NU_M)
    assert e.value.code == hom.HOM_EINVAL
    with pytest.raises(hom.HomError):
        hom.hom_create(phi.shape, phi, hom.HOM_INPUT_FRACTION_F64, -1.0, NU_M)
    with make(hom, phi, "fp32") as ctx:
        rc, info = hom.hom_solve(ctx, np.eye(6)[0], tol=1e-12, max_it=2)
        assert rc == hom.HOM_NOT_CONVERGED and info[0]["status"] == hom.HOM_NOT_CONVERGED
        with pytest.raises(hom.HomError):
            hom.hom_effective_stiffness(ctx)       # fewer than 6 cases
        with pytest.raises(hom.HomError):
            hom.hom_fields(ctx, 3)


def test_largest_axis_and_device_pointers(hom):
    """n = 512 on one axis (largest supported transform) and device buffers."""
    import torch
    shape = (4, 6, 512)
    phi = ri.random_phi(shape, seed=4)
    f = ri.random_field(shape, seed=5)
    ctx = hom.hom_create(shape, torch.tensor(phi, device="cuda"), hom.HOM_INPUT_FRACTION_F64, E_M, NU_M,
                         precision=hom.HOM_PREC_FP32_FIELDS, device_ptrs=True)
    try:
        fin = torch.tensor(f, dtype=torch.float32, device="cuda")
        out = torch.empty_like(fin)
        hom.hom_apply(ctx, fin, out)
        torch.cuda.synchronize()
        ref = oracle.apply(phi, 1.0, NU_M, 1, f)
        assert rel_maxerr(out.cpu().numpy(), ref) <= FP32_TOL
        shape2 = (512, 4, 6)
        phi2 = ri.random_phi(shape2, seed=6)
        with make(hom, phi2, "fp32") as c2:
            g = hom.hom_apply(c2, f.reshape((6,) + shape2).astype(np.float32))
            assert rel_maxerr(g, oracle.apply(phi2, 1.0, NU_M, 1, f.reshape((6,) + shape2))) <= FP32_TOL
    finally:
        ctx.close()


def test_tma_staging_matches_plain_loads(hom):
    """The persistent TMA-staged n1/n2 passes compute exactly what the plain-
    load passes compute (same FFT code, different data movement)."""
    shape = (256, 128, 16)
    phi = ri.random_phi(shape, seed=8)
    f = ri.random_field(shape, seed=9).astype(np.float32)
    outs = []
    for staging in (0, 1):
        with hom.hom_create(shape, phi, hom.HOM_INPUT_FRACTION_F64, E_M, NU_M, staging=staging) as ctx:
            outs.append(hom.hom_apply(ctx, f))
            spec = hom.hom_fft_forward(ctx, f)
            outs.append(spec)
    assert np.array_equal(outs[0], outs[2])
    assert np.array_equal(outs[1], outs[3])


def test_solve_tma_octet_matches_oracle(hom):
    """FP32 solve on a grid whose n1/n2 passes are TMA-staged (64^3 octet)."""
    phi, _ = ri.octet(64, 0.2)
    phi = phi.astype(np.float64)
    Eb = np.array([1.0, 0, 0, 0, 0, 0])
    ref = oracle.solve(phi, E_M, NU_M, 1, Eb, tol=1e-10, max_it=6000)
    assert ref["true_residual"] < 1e-9
    with make(hom, phi, "fp32") as ctx:
        rc, info = hom.hom_solve(ctx, Eb, tol=1e-7, max_it=6000)
        assert rc == hom.HOM_OK, info
        err = np.max(np.abs(info[0]["sigma_mean"] - ref["sigma_mean"])) / np.max(np.abs(ref["sigma_mean"]))
        assert err <= 1e-4, err


# Transform lengths of the 256^3 headline and of the 512^3 as-printed run:
# length 256 on n3 (register engine, the headline's n3 pass) beside TMA-staged
# n1/n2 passes of length 64; length 256 on the TMA-staged n1 pass; n1 = n2 =
# 256 (both TMA-staged, as at 256^3); length 512 on n2 and on n1 in plain-
# load passes (the other axis short) and in TMA-staged ones (the other axis
# 64), as the 512^3 cell takes them.
LONG_SHAPES = [(64, 64, 256), (256, 64, 64), (256, 256, 8), (8, 512, 8), (512, 8, 16), (512, 64, 8), (64, 512, 8)]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("shape", LONG_SHAPES)
def test_long_axes_fft(hom, shape, prec):
    test_fft_forward_inverse(hom, shape, prec)


@pytest.mark.parametrize("deriv", [0, 1])
@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("shape", LONG_SHAPES)
def test_long_axes_project_apply_rhs(hom, shape, prec, deriv):
    test_project_apply_rhs(hom, shape, prec, deriv)


def _golden(name):
    import json
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", name)
    with open(path) as f:
        return json.load(f)


@pytest.mark.parametrize("tol", [1e-6, 1e-7])
def test_solve_octet128_matches_stored_oracle(hom, tol):
    """128^3 octet at density 0.10 (the headline cell at half the resolution):
    the FP32-field solve's mean stress of E11 and E23 against the FP64
    oracle's, solved to 1e-10 and stored by tests/golden/make_octet_golden.py,
    within 1e-4 of the largest entry -- the effective-stiffness columns of
    section 4.3.  At tol 1e-6 (the headline tolerance) as well as 1e-7."""
    gold = _golden("octet128_rho0.10.json")
    phi, radius = ri.octet(128, gold["relative_density"])
    assert abs(radius - gold["radius"]) < 1e-12 and abs(phi.mean() - gold["phi_mean"]) < 1e-6
    macro = np.array([c["macro_strain"] for c in gold["cases"]])
    with make(hom, phi.astype(np.float64), "fp32") as ctx:
        rc, info = hom.hom_solve(ctx, macro, tol=tol, max_it=5000)
        assert rc == hom.HOM_OK, [i["status"] for i in info]
        for case, inf in zip(gold["cases"], info):
            ref = np.array(case["sigma_mean"])
            err = np.max(np.abs(np.array(inf["sigma_mean"]) - ref)) / np.max(np.abs(ref))
            assert err <= 1e-4, (case["macro_strain"], err)
            assert inf["true_residual"] <= tol


# the spectral operator the MINRES iteration applies; n3 in {64, 128, 256}
# runs the register-resident n3 pass in FP32, the others the shared-memory one
SPEC_SHAPES = [(16, 8, 64), (8, 12, 128), (64, 64, 256), (12, 10, 9), (32, 32, 32), (6, 4, 256)]


@pytest.mark.parametrize("deriv", [0, 1])
@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("shape", SPEC_SHAPES)
def test_apply_spectrum(hom, shape, prec, deriv):
    """G F C F^-1 G on the DFT of a field equals the DFT of the oracle's
    A(G e), eq. (linearOp) with the projector of eq. (galop) on the input."""
    phi = ri.random_phi(shape, seed=12)
    f = ri.random_field(shape, seed=13)
    spec_in = np.moveaxis(half_spectrum(np.stack([oracle.fft3d(f[c].astype(complex)) for c in range(6)])), 0, -1)
    ref_real = oracle.apply(phi, 1.0, NU_M, deriv, oracle.project(shape, deriv, f))
    ref = np.moveaxis(half_spectrum(np.stack([oracle.fft3d(ref_real[c].astype(complex)) for c in range(6)])), 0, -1)
    with make(hom, phi, prec, deriv) as ctx:
        cdt = np.complex64 if prec == "fp32" else np.complex128
        got = hom.hom_apply_spectrum(ctx, np.ascontiguousarray(spec_in.astype(cdt)))
        assert rel_maxerr(got, ref) <= tol(prec)


# the mixed register-FFT plans 96 = 4 4 2 3 and 160 = 4 4 2 5 (the batched
# cell studies' grids) on every axis: TMA-staged n1 / n2 passes in FP32
# where both are 96 or 160, plain passes otherwise, and the n3 pass
MIXED_SHAPES = [(96, 96, 8), (160, 160, 6), (160, 96, 10), (8, 6, 160), (10, 8, 96), (96, 4, 160)]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("shape", MIXED_SHAPES)
def test_mixed_plans_fft(hom, shape, prec):
    test_fft_forward_inverse(hom, shape, prec)


@pytest.mark.parametrize("deriv", [0, 1])
@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("shape", MIXED_SHAPES)
def test_mixed_plans_project_apply_rhs(hom, shape, prec, deriv):
    test_project_apply_rhs(hom, shape, prec, deriv)


@pytest.mark.parametrize("shape", [(96, 96, 8), (160, 160, 6), (8, 6, 160)])
def test_mixed_plans_apply_spectrum(hom, shape):
    test_apply_spectrum(hom, shape, "fp32", 1)


def test_solve_octet256_headline_matches_stored_oracle(hom):
    """The 256^3 headline cell (octet, density 0.10, E11, tol 1e-6, FP32
    fields): mean stress against the FP64 oracle's, solved to 1e-10 and stored
    by tests/golden/make_octet_golden.py, within 1e-4 of its largest entry."""
    gold = _golden("octet256_rho0.10.json")
    phi, radius = ri.octet(256, gold["relative_density"])
    assert abs(radius - gold["radius"]) < 1e-12
    case = gold["cases"][0]
    with make(hom, phi.astype(np.float64), "fp32") as ctx:
        rc, info = hom.hom_solve(ctx, np.array(case["macro_strain"]), tol=1e-6, max_it=5000)
        assert rc == hom.HOM_OK
        ref = np.array(case["sigma_mean"])
        err = np.max(np.abs(np.array(info[0]["sigma_mean"]) - ref)) / np.max(np.abs(ref))
        assert err <= 1e-4, err
        assert info[0]["true_residual"] <= 1e-6


@pytest.mark.parametrize("prec", PRECS)
def test_laminate_512_axis(hom, prec):
    """Layered cell with n1 = 512 and n2 = 64: the MINRES solve through the
    TMA-staged n1 pass of length 512 (two 256-row boxes per tile) in FP32,
    against the exact laminate closed form."""
    from test_oracle_solver import laminate_closed_form
    phi = ri.laminate((512, 64, 8), (256, 128, 128), (1.0, 0.2, 0.55), axis=0)
    with make(hom, phi, prec) as ctx:
        rc, info = hom.hom_solve(ctx, np.eye(6), tol=1e-9, max_it=500)
        assert rc == hom.HOM_OK
        for J in range(6):
            ref = laminate_closed_form([1.0, 0.2, 0.55], [0.5, 0.25, 0.25], np.eye(6)[J])
            assert np.allclose(info[J]["sigma_mean"], ref, rtol=1e-5, atol=1e-5 * E_M)


@pytest.mark.parametrize("shape,thick", [((96, 64, 8), (48, 24, 24)), ((160, 64, 8), (80, 40, 40)),
                                         ((64, 96, 8), (32, 16, 16))])
def test_laminate_mixed_n1_fused_step(hom, shape, thick):
    """Layered cells whose n1 is 96 or 160 (mixed register plans) with a
    register-length n2: FP32 solves through the warp-specialised fused n1
    pass, whose lagged-update items do not divide its Krylov blocks evenly
    (18 and 30 KB per tile against 4 KB items), against the exact laminate
    closed form (layers normal to e1, section 4's periodic setting)."""
    from test_oracle_solver import laminate_closed_form
    n1 = shape[0]
    fr = [t / n1 for t in thick]
    phi = ri.laminate(shape, thick, (1.0, 0.2, 0.55), axis=0)
    with make(hom, phi, "fp32") as ctx:
        rc, info = hom.hom_solve(ctx, np.eye(6), tol=1e-9, max_it=800)
        assert rc == hom.HOM_OK
        for J in range(6):
            ref = laminate_closed_form([1.0, 0.2, 0.55], fr, np.eye(6)[J])
            assert np.allclose(info[J]["sigma_mean"], ref, rtol=1e-5, atol=1e-5 * E_M)
            assert info[J]["true_residual"] <= 1e-9
