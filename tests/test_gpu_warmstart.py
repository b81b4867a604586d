"""hom_solve from a given initial strain (the warm-start hook of the learned
initial iterate; the paper restarts Newton steps from the previous strain,
section 2.1.1).  The start is projected onto compatible fields and the FP64
true residual decides convergence, so any start gives the zero-start answer."""
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
def test_warm_start_from_solution_and_from_perturbed_solution(hom, prec):
    p = hom.HOM_PREC_FP32_FIELDS if prec == "fp32" else hom.HOM_PREC_FP64
    dt = np.float32 if prec == "fp32" else np.float64
    phi, _ = ri.octet(32, 0.15)
    E = np.array([[1e-3, 0, 0, 0, 0, 0], [0, 0, 0, 5e-4, 0, 0]])
    with hom.hom_create(phi.shape, phi, hom.HOM_INPUT_FRACTION_F32, E_M, NU_M, precision=p) as ctx:
        rc, zero = hom.hom_solve(ctx, E, tol=1e-7, max_it=5000)
        assert rc == hom.HOM_OK
        fluct = []
        for k in range(2):
            strain, _ = hom.hom_fields(ctx, k, want=("strain",))
            fluct.append(strain - E[k][:, None, None, None])
        exact = np.ascontiguousarray(np.stack(fluct), dtype=dt)
        rc, warm = hom.hom_solve(ctx, E, tol=1e-7, max_it=5000, warm_start=exact)
        assert rc == hom.HOM_OK
        for k in range(2):
            assert warm[k]["iterations"] <= max(5, zero[k]["iterations"] // 10), (warm[k], zero[k])
            ref = zero[k]["sigma_mean"]
            assert np.max(np.abs(warm[k]["sigma_mean"] - ref)) <= 1e-6 * np.max(np.abs(ref))
        rng = np.random.default_rng(3)
        noisy = np.ascontiguousarray(exact * (1 + 0.2 * rng.standard_normal(exact.shape)), dtype=dt)
        rc, pert = hom.hom_solve(ctx, E, tol=1e-7, max_it=5000, warm_start=noisy)
        assert rc == hom.HOM_OK
        for k in range(2):
            assert pert[k]["true_residual"] <= 1e-7
            ref = zero[k]["sigma_mean"]
            assert np.max(np.abs(pert[k]["sigma_mean"] - ref)) <= 1e-5 * np.max(np.abs(ref))
