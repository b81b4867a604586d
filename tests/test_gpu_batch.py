"""Batched solves over cells of different sizes, and the launch-shape autotuner."""
import numpy as np
import pytest

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


def test_batch_equals_one_by_one(hom):
    cells = [(16, 0.25), (24, 0.12), (32, 0.05)]      # power-of-two and mixed-radix grids
    macros = np.array([np.eye(6)[0], np.eye(6)[4]]) * 1e-3
    ctxs = []
    for n, rho in cells:
        phi, _ = ri.octet(n, rho)
        ctxs.append(hom.hom_create(phi.shape, phi, hom.HOM_INPUT_FRACTION_F32, E_M, NU_M))
    rc, infos = hom.hom_solve_batch(ctxs, macros, tol=1e-7, max_it=5000)
    assert rc == hom.HOM_OK
    batch = [[i["sigma_mean"] for i in cell] for cell in infos]
    for c, ctx in enumerate(ctxs):
        rc1, one = hom.hom_solve(ctx, macros, tol=1e-7, max_it=5000)
        assert rc1 == hom.HOM_OK
        for k in range(len(macros)):
            assert np.array_equal(batch[c][k], one[k]["sigma_mean"])
        ctx.close()


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
