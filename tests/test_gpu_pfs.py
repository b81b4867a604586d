"""GPU parity of the phase-field smoothening (hom_pfs; section 3.2) against
the FP64 oracle: the filtered, block-averaged, thresholded phase map element
by element (FP64 FFTs on both sides, 1e-12), for cubic and non-cubic fine
grids, float and byte indicators, host and device buffers; the conservation
of the mean without threshold; the rejections; and a solve on the result."""
import numpy as np
import pytest

import oracle
import rve_inputs as ri

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hom():
    import torch
    assert torch.cuda.is_available()
    from paper_2110_00733_gb300 import build, hom as h
    build.build()
    h.load_library()
    return h


def indicator(shape, rho=0.2):
    n = shape[0]
    phi, _ = ri.octet(shape if len(set(shape)) > 1 else n, rho)
    return (phi >= 0.5)


@pytest.mark.parametrize("shape,ratio,ell", [((32, 32, 32), 2, 1.0), ((24, 18, 30), 3, 1.5), ((40, 40, 40), 4, 2.0)])
def test_pfs_matches_oracle(hom, shape, ratio, ell):
    omega = indicator(shape).astype(np.float64)
    ref = oracle.pfs(omega, ratio, ell, 1.0, 0.05)
    got = hom.hom_pfs(omega, ratio, ell, 1.0, 0.05)
    assert got.shape == ref.shape
    # the threshold may only differ where the unthresholded value sits within
    # round-off of it
    raw = oracle.pfs(omega, ratio, ell, 1.0, 0.0)
    near = np.abs(raw - 0.05) < 1e-12
    assert np.max(np.abs(got - ref)[~near]) <= 1e-12


def test_pfs_byte_input_and_device_buffers(hom):
    import torch
    shape = (32, 32, 32)
    om = indicator(shape).astype(np.uint8)
    ref = oracle.pfs(om.astype(np.float64), 2, 1.0, 1.0, 0.05)
    got = hom.hom_pfs(om, 2, 1.0, 1.0, 0.05)
    assert np.max(np.abs(got - ref)) <= 1e-12
    dev_in = torch.from_numpy(om.astype(np.float32)).cuda()
    dev_out = torch.zeros((16, 16, 16), dtype=torch.float64, device="cuda")
    hom.hom_pfs(dev_in, 2, 1.0, 1.0, 0.05, out=dev_out)
    assert np.max(np.abs(dev_out.cpu().numpy() - ref)) <= 1e-12


def test_pfs_conserves_the_mean_without_threshold(hom):
    omega = indicator((48, 48, 48)).astype(np.float64)
    got = hom.hom_pfs(omega, 3, 1.5, 1.0, 0.0)
    assert got.mean() == pytest.approx(omega.mean(), rel=1e-12)


def test_pfs_rejections_and_a_solve_on_its_map(hom):
    omega = indicator((32, 32, 32)).astype(np.float64)
    with pytest.raises(hom.HomError) as e:
        hom.hom_pfs(omega, 3, 1.0)                        # 32 is not a multiple of 3
    assert e.value.code == hom.HOM_EINVAL
    with pytest.raises(hom.HomError) as e:
        hom.hom_pfs(omega, 2, -1.0)
    assert e.value.code == hom.HOM_EINVAL
    phi = hom.hom_pfs(omega, 2, 1.0)
    with hom.hom_create(phi.shape, phi, hom.HOM_INPUT_FRACTION_F64, 110e9, 0.3) as ctx:
        rc, info = hom.hom_solve(ctx, np.eye(6)[[0]], tol=1e-6, max_it=3000)
        assert rc == hom.HOM_OK and info[0]["sigma_mean"][0] > 0
