"""Batched solves over cells of different sizes and stacked load cases,
checked against the FP64 oracle, and the launch-shape autotuner."""
import numpy as np
import pytest

import oracle
import rve_inputs as ri
from gpu_util import FP32_TOL

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


def test_batch_matches_oracle(hom):
    """Cells of different sizes (power-of-two and mixed-radix grids, different
    densities) solved at once by hom_solve_batch, each with its six unit macro
    strains stacked in one launch: the effective stiffness of every cell
    against the FP64 oracle's (section 4.3), within 1e-4 of its largest
    entry."""
    cells = [(16, 0.25), (24, 0.12), (32, 0.05)]
    ctxs, refs = [], []
    for n, rho in cells:
        phi, _ = ri.octet(n, rho)
        ctxs.append(hom.hom_create(phi.shape, phi, hom.HOM_INPUT_FRACTION_F32, E_M, NU_M))
        Cref, _ = oracle.effective_stiffness(phi.astype(np.float64), E_M, NU_M, 1, tol=1e-10, max_it=20000)
        refs.append(Cref)
    try:
        rc, infos = hom.hom_solve_batch(ctxs, np.eye(6), tol=1e-8, max_it=20000)
        assert rc == hom.HOM_OK, [[i["status"] for i in cell] for cell in infos]
        for ctx, Cref, cell in zip(ctxs, refs, infos):
            C = hom.hom_effective_stiffness(ctx)
            assert np.max(np.abs(C - Cref)) <= 1e-4 * np.max(np.abs(Cref))
            assert all(i["true_residual"] <= 1e-8 for i in cell)
    finally:
        for c in ctxs:
            c.close()


def test_stacked_cases_match_one_at_a_time(hom):
    """The six load cases stacked in one launch give what each case gives on
    its own (same kernels, so agreement to FP32 round-off of the solve)."""
    phi, _ = ri.octet(24, 0.15)
    macros = np.eye(6) * 1e-3
    with hom.hom_create(phi.shape, phi, hom.HOM_INPUT_FRACTION_F32, E_M, NU_M) as ctx:
        rc, together = hom.hom_solve(ctx, macros, tol=1e-8, max_it=5000)
        assert rc == hom.HOM_OK
        for k in range(6):
            rc, alone = hom.hom_solve(ctx, macros[k], tol=1e-8, max_it=5000)
            assert rc == hom.HOM_OK
            ref = np.asarray(alone[0]["sigma_mean"])
            assert np.max(np.abs(np.asarray(together[k]["sigma_mean"]) - ref)) <= 1e-6 * np.max(np.abs(ref))


def test_autotune_shapes_give_the_same_answer(hom):
    shape = (64, 64, 64)
    tuned = hom.hom_autotune(shape)
    assert len(tuned) == 3 and all(v >= 0 for v in tuned)
    assert hom.hom_autotune(shape) == tuned                 # cached
    phi, _ = ri.octet(64, 0.15)
    f = ri.random_field(shape, seed=31).astype(np.float32)
    with hom.hom_create(shape, phi, hom.HOM_INPUT_FRACTION_F32, E_M, NU_M) as c0, \
            hom.hom_create(shape, phi, hom.HOM_INPUT_FRACTION_F32, E_M, NU_M, autotune=True) as c1:
        a0 = hom.hom_apply(c0, f)
        a1 = hom.hom_apply(c1, f)
        assert np.max(np.abs(a0 - a1)) <= FP32_TOL * np.max(np.abs(a0))


def test_batch_of_laminates_on_the_fused_kernels(hom):
    """Two layered cells at sizes that take the fused MINRES step (TMA-staged
    n1 / n2 passes, the warp-specialised n1 pass with its lagged-update ring
    and deferred x update, the persistent register n3 pass at n3 = 64 and the
    two-stage shared-memory n3 pass at n3 = 96), solved together by
    hom_solve_batch with the six unit strains stacked: every mean stress
    against the exact laminate closed form (layers normal to e1)."""
    from test_oracle_solver import laminate_closed_form
    vals = (1.0, 0.2, 0.55)
    cells = [((64, 64, 64), (32, 16, 16)), ((96, 64, 96), (48, 24, 24))]
    ctxs = []
    for shape, thick in cells:
        phi = ri.laminate(shape, thick, vals, axis=0)
        ctxs.append(hom.hom_create(phi.shape, phi.astype(np.float32), hom.HOM_INPUT_FRACTION_F32, E_M, NU_M))
    try:
        rc, infos = hom.hom_solve_batch(ctxs, np.eye(6), tol=1e-9, max_it=2000)
        assert rc == hom.HOM_OK, [[i["status"] for i in cell] for cell in infos]
        for (shape, thick), cell in zip(cells, infos):
            fr = [t / shape[0] for t in thick]
            for J in range(6):
                ref = laminate_closed_form(list(vals), fr, np.eye(6)[J])
                assert np.allclose(cell[J]["sigma_mean"], ref, rtol=1e-5, atol=1e-5 * E_M), (shape, J)
                assert cell[J]["true_residual"] <= 1e-9
    finally:
        for c in ctxs:
            c.close()


def test_stacked_cases_match_one_at_a_time_64(hom):
    """The same at 64^3, where the persistent register n3 pass and the
    warp-specialised n1 pass run (cases that converge at different steps are
    skipped by those kernels while the others go on)."""
    phi, _ = ri.octet(64, 0.15)
    macros = np.eye(6) * 1e-3
    with hom.hom_create(phi.shape, phi, hom.HOM_INPUT_FRACTION_F32, E_M, NU_M) as ctx:
        rc, together = hom.hom_solve(ctx, macros, tol=1e-8, max_it=5000)
        assert rc == hom.HOM_OK
        its = {i["iterations"] for i in together}
        for k in range(6):
            rc, alone = hom.hom_solve(ctx, macros[k], tol=1e-8, max_it=5000)
            assert rc == hom.HOM_OK
            ref = np.asarray(alone[0]["sigma_mean"])
            assert np.max(np.abs(np.asarray(together[k]["sigma_mean"]) - ref)) <= 1e-6 * np.max(np.abs(ref))
        assert len(its) > 1   # the cases did converge at different steps
