"""hom_apply_noalloc: the allocation-free entry point for callers that must
not call cudaMalloc (an application whose device memory belongs to its own
pool or is reserved up front, or a latency-critical loop in which cudaMalloc,
which may synchronise the device, is not acceptable).

Checked through the C ABI against the existing hom_apply entry point, within
the FP32 parity tolerance, on two calls in a row (the scratch arrays are
shared by every call and keep the previous call's contents), and against the
FP64 oracle's A(eps) of eq. (linearOp) for both derivative schemes, on the
legacy default stream, on a side stream and recorded in a CUDA graph.  The
call only enqueues its kernels, so each check synchronises before reading the
output.  This file is
collected last so that a run stopping at the first failure has already run
every other test."""
import numpy as np
import pytest

import oracle
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
            torch.cuda.synchronize()
            hom.hom_apply_noalloc(shape, phi_d, eps, out, E=E_M, nu=NU_M)
            torch.cuda.synchronize()
            got = out.cpu().numpy()
            assert np.all(np.isfinite(got))
            assert rel_maxerr(got, ref) <= FP32_TOL


@pytest.mark.parametrize("side_stream", [False, True])
@pytest.mark.parametrize("deriv", [0, 1])
@pytest.mark.parametrize("shape", [(32, 24, 20), (64, 16, 32)])
def test_noalloc_matches_oracle(hom, shape, deriv, side_stream):
    """A(eps) against the oracle; (64, 16, 32) runs the register FFT of length
    64 on n1 and 32 on n3, (32, 24, 20) the generic mixed-radix engine on n2."""
    import torch
    phi = ri.random_phi(shape, seed=31).astype(np.float32)
    f = ri.random_field(shape, seed=32)
    ref = oracle.apply(phi.astype(np.float64), 1.0, NU_M, deriv, f)   # units of E, like the entry point
    phi_d = torch.tensor(phi, device="cuda")
    eps = torch.tensor(f, dtype=torch.float32, device="cuda")
    out = torch.full_like(eps, float("nan"))
    torch.cuda.synchronize()
    if side_stream:
        s = torch.cuda.Stream()
        hom.hom_apply_noalloc(shape, phi_d, eps, out, E=E_M, nu=NU_M, derivative=deriv, stream=s.cuda_stream)
        s.synchronize()
    else:
        hom.hom_apply_noalloc(shape, phi_d, eps, out, E=E_M, nu=NU_M, derivative=deriv)
        torch.cuda.synchronize()
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


@pytest.mark.parametrize("deriv", [0, 1])
def test_noalloc_recorded_in_a_cuda_graph(hom, deriv):
    """The call records into a CUDA graph (it enqueues kernels only and does
    not wait on the stream): one eager call first makes the per-device set-up,
    then the call is captured on torch's capture stream and replayed on new
    contents of the same input buffer; each replay is compared with the oracle."""
    import torch
    shape = (64, 16, 32)
    phi = ri.random_phi(shape, seed=41).astype(np.float32)
    phi_d = torch.tensor(phi, device="cuda")
    eps = torch.zeros((6,) + shape, dtype=torch.float32, device="cuda")
    out = torch.full_like(eps, float("nan"))
    hom.hom_apply_noalloc(shape, phi_d, eps, out, E=E_M, nu=NU_M, derivative=deriv)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        hom.hom_apply_noalloc(shape, phi_d, eps, out, E=E_M, nu=NU_M, derivative=deriv,
                              stream=torch.cuda.current_stream().cuda_stream)
    for seed in (42, 43):
        f = ri.random_field(shape, seed=seed)
        eps.copy_(torch.tensor(f, dtype=torch.float32))
        out.fill_(float("nan"))
        graph.replay()
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        ref = oracle.apply(phi.astype(np.float64), 1.0, NU_M, deriv, f)
        assert np.all(np.isfinite(got))
        assert rel_maxerr(got, ref) <= FP32_TOL
