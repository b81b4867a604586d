"""Degenerate inputs of the solver on the GPU: an all-empty cell, grid sizes
outside the supported range, a binary phase map given as uint8, max_it = 0,
and the MoDBFFT solver on a homogeneous cell."""
import numpy as np
import pytest

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


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_empty_cell_has_zero_stiffness(hom, prec):
    """phi = 0 everywhere: C : E_bar = 0, so b = 0, zero iterations and
    C_eff = 0 exactly."""
    p = hom.HOM_PREC_FP32_FIELDS if prec == "fp32" else hom.HOM_PREC_FP64
    phi = np.zeros((8, 12, 10), dtype=np.float32)
    with hom.hom_create(phi.shape, phi, hom.HOM_INPUT_FRACTION_F32, E_M, NU_M, precision=p) as ctx:
        rc, info = hom.hom_solve(ctx, np.eye(6), tol=1e-6, max_it=100)
        assert rc == hom.HOM_OK and all(i["iterations"] == 0 for i in info)
        assert np.array_equal(hom.hom_effective_stiffness(ctx), np.zeros((6, 6)))


@pytest.mark.parametrize("grid", [(0, 8, 8), (1, 8, 8), (8, 8, 513), (8, 7, 8)])
def test_unsupported_grids_are_rejected(hom, grid):
    phi = np.ones(max(1, int(np.prod(grid))), dtype=np.float32)
    with pytest.raises(hom.HomError) as e:
        hom.hom_create(grid, phi, hom.HOM_INPUT_FRACTION_F32, E_M, NU_M)
    assert e.value.code == hom.HOM_EUNSUPPORTED_GRID


def test_uint8_phase_equals_binary_fraction(hom):
    """A uint8 phase map (0 empty, nonzero solid) solves like the same map
    given as 0/1 fractions."""
    phi, _ = ri.octet(16, 0.2)
    binary = (phi >= 0.5)
    u8 = np.ascontiguousarray(binary.astype(np.uint8) * 3)
    E = np.eye(6)[[0, 3]]
    with hom.hom_create(u8.shape, u8, hom.HOM_INPUT_PHASE_U8, E_M, NU_M) as a, \
            hom.hom_create(u8.shape, binary.astype(np.float32), hom.HOM_INPUT_FRACTION_F32, E_M, NU_M) as b:
        _, ia = hom.hom_solve(a, E, tol=1e-7, max_it=5000)
        _, ib = hom.hom_solve(b, E, tol=1e-7, max_it=5000)
        for x, y in zip(ia, ib):
            assert np.array_equal(x["sigma_mean"], y["sigma_mean"])


def test_zero_iteration_budget_reports_the_start_residual(hom):
    phi, _ = ri.octet(16, 0.2)
    with hom.hom_create(phi.shape, phi, hom.HOM_INPUT_FRACTION_F32, E_M, NU_M) as ctx:
        rc, info = hom.hom_solve(ctx, np.eye(6)[0], tol=1e-6, max_it=0)
        assert rc == hom.HOM_NOT_CONVERGED
        assert info[0]["iterations"] == 0
        assert info[0]["true_residual"] == pytest.approx(1.0)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_modbfft_homogeneous_cell(hom, prec):
    """MoDBFFT on phi = 1: the right-hand side is zero, C_eff = C_m."""
    from test_oracle_solver import voigt_stiffness
    p = hom.HOM_PREC_FP32_FIELDS if prec == "fp32" else hom.HOM_PREC_FP64
    phi = np.ones((8, 8, 12), dtype=np.float32)
    with hom.hom_create(phi.shape, phi, hom.HOM_INPUT_FRACTION_F32, E_M, NU_M, derivative=hom.HOM_DERIV_CONTINUOUS,
                        precision=p, solver=hom.HOM_SOLVER_MODBFFT_CG) as ctx:
        rc, info = hom.hom_solve(ctx, np.eye(6), tol=1e-8, max_it=100)
        assert rc == hom.HOM_OK and all(i["iterations"] == 0 for i in info)
        assert np.allclose(hom.hom_effective_stiffness(ctx), voigt_stiffness(E_M, NU_M), rtol=1e-9)


def test_host_replayed_loop_matches_device_loop(hom):
    """host_loop replays the same captured body from the host: the same
    kernels in the same order give the same iterates, so iteration counts and
    stresses agree exactly."""
    phi, _ = ri.octet(32, 0.15)
    E = np.eye(6)[[0, 3]]
    out = []
    for host_loop in (False, True):
        with hom.hom_create(phi.shape, phi, hom.HOM_INPUT_FRACTION_F32, E_M, NU_M, host_loop=host_loop) as ctx:
            rc, info = hom.hom_solve(ctx, E, tol=1e-6, max_it=5000)
            assert rc == hom.HOM_OK
            out.append(info)
    for a, b in zip(*out):
        assert a["iterations"] == b["iterations"]
        assert np.array_equal(a["sigma_mean"], b["sigma_mean"])
