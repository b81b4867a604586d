"""hom_apply_noalloc: the allocation-free entry point for callers that must
not call cudaMalloc (a thread recording a CUDA graph by stream capture, or an
application whose device memory belongs to its own pool).

Checked through the C ABI against the existing hom_apply entry point, within
the FP32 parity tolerance, on two calls in a row (the scratch arrays are
shared by every call and keep the previous call's contents).  This file is
collected last so that a run stopping at the first failure has already run
every other test."""
import numpy as np
import pytest

import rve_inputs as ri
from gpu_util import FP32_TOL, rel_maxerr

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


def test_noalloc_matches_hom_apply_twice(hom):
    import torch
    shape = (32, 24, 20)
    phi = ri.random_phi(shape, seed=21).astype(np.float32)
    phi_d = torch.tensor(phi, device="cuda")
    with hom.hom_create(shape, phi, hom.HOM_INPUT_FRACTION_F32, E_M, NU_M) as ctx:
        for seed in (22, 23):            # two calls in a row, different inputs
            f = ri.random_field(shape, seed=seed).astype(np.float32)
            ref = hom.hom_apply(ctx, f)
            eps = torch.tensor(f, device="cuda")
            out = torch.full_like(eps, float("nan"))
            hom.hom_apply_noalloc(shape, phi_d, eps, out, E=E_M, nu=NU_M)
            got = out.cpu().numpy()
            assert np.all(np.isfinite(got))
            assert rel_maxerr(got, ref) <= FP32_TOL


def test_noalloc_rejects_grids_beyond_the_limit(hom):
    import torch
    shape = (64, 32, 20)                 # 40960 voxels > 32768
    phi = torch.zeros(shape, device="cuda")
    eps = torch.zeros((6,) + shape, device="cuda")
    with pytest.raises(hom.HomError) as e:
        hom.hom_apply_noalloc(shape, phi, eps, torch.empty_like(eps))
    assert e.value.code == hom.HOM_EUNSUPPORTED_GRID
    assert "32768" in hom.hom_last_error(None)
