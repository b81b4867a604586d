"""Pins of the warm-start network oracle against library routines, adjoint
identities, finite differences and structural invariants."""
import numpy as np
import pytest

from oracle import net_oracle as no

SMALL = (2, 3, 2, 3)          # channel widths small enough for finite differences


def test_conv_matches_scipy_wrap_correlation():
    ndimage = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(0)
    x = rng.standard_normal((1, 5, 6, 7, 2))
    W = rng.standard_normal((27, 3, 2))
    b = rng.standard_normal(3)
    y = no.conv3d(x, W, b)
    for co in range(3):
        ref = b[co] + sum(ndimage.correlate(x[0, ..., ci], W[:, co, ci].reshape(3, 3, 3), mode="wrap")
                          for ci in range(2))
        assert np.allclose(y[0, ..., co], ref, atol=1e-12)


def test_dgrad_and_wgrad_are_adjoints():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((2, 4, 6, 4, 3))
    W = rng.standard_normal((27, 5, 3))
    g = rng.standard_normal((2, 4, 6, 4, 5))
    lhs = np.sum(no.conv3d(x, W, np.zeros(5)) * g)
    assert np.isclose(lhs, np.sum(x * no.conv3d_dgrad(g, W)), rtol=1e-12)
    dW, db = no.conv3d_wgrad(g, x)
    assert np.isclose(lhs, np.sum(W * dW), rtol=1e-12)
    assert np.allclose(db, g.sum(axis=(0, 1, 2, 3)))


def test_pool_and_upsample_adjoints():
    rng = np.random.default_rng(2)
    a = rng.standard_normal((1, 2, 3, 2, 4))
    f = rng.standard_normal((1, 4, 6, 4, 4))
    assert np.isclose(np.sum(no.upsample2(a) * f), np.sum(a * no.upsample2_grad(f)))
    assert np.isclose(np.sum(no.avgpool2(f) * a), np.sum(f * no.avgpool2_grad(a)))
    assert np.allclose(no.avgpool2(no.upsample2(a)), a)


def _tiny(seed=3, n=8, B=2):
    rng = np.random.default_rng(seed)
    specs = no.layer_specs(SMALL)
    P = no.init_params(specs, rng)
    for k in P:                                  # non-zero biases and a visible head
        P[k] = P[k] + 0.05 * rng.standard_normal(P[k].shape)
    phi = rng.random((B, n, n, n))
    E = rng.standard_normal((B, 6))
    target = rng.standard_normal((B, n, n, n, 6))
    return specs, P, phi, E, target


def _loss(specs, P, phi, E, target):
    x0, _ = no.forward(P, phi, E, specs)
    return no.loss_and_grad_out(x0, target)[0]


def test_backward_matches_finite_differences():
    specs, P, phi, E, target = _tiny()
    x0, cache = no.forward(P, phi, E, specs)
    _, gx = no.loss_and_grad_out(x0, target)
    G = no.backward(P, cache, gx, specs)
    rng = np.random.default_rng(4)
    h = 1e-6
    for name, *_ in specs:
        for key in (name + ".W", name + ".b"):
            for _ in range(3):
                idx = tuple(rng.integers(0, s) for s in P[key].shape)
                old = P[key][idx]
                P[key][idx] = old + h
                lp = _loss(specs, P, phi, E, target)
                P[key][idx] = old - h
                lm = _loss(specs, P, phi, E, target)
                P[key][idx] = old
                fd = (lp - lm) / (2 * h)
                assert abs(fd - G[key][idx]) <= 1e-6 * max(1e-3, abs(fd)), (key, idx, fd, G[key][idx])


def test_prediction_is_linear_in_macro_strain_and_shift_equivariant():
    specs, P, phi, E, _ = _tiny(n=16, B=1)
    E2 = np.random.default_rng(5).standard_normal((1, 6))
    a, b = 0.7, -1.3
    x1, _ = no.forward(P, phi, E, specs)
    x2, _ = no.forward(P, phi, E2, specs)
    x3, _ = no.forward(P, phi, a * E + b * E2, specs)
    assert np.allclose(x3, a * x1 + b * x2, atol=1e-12)
    # three 2x poolings: shifts by multiples of 8 voxels commute with the network
    xs, _ = no.forward(P, np.roll(phi, (8, 0, 8), axis=(1, 2, 3)), E, specs)
    assert np.allclose(xs, np.roll(x1, (8, 0, 8), axis=(1, 2, 3)), atol=1e-12)


def test_adam_first_step_is_signed_learning_rate():
    P = {"w": np.array([1.0, -2.0, 0.5])}
    G = {"w": np.array([3e-2, -4e-4, 0.0])}
    m = {"w": np.zeros(3)}
    v = {"w": np.zeros(3)}
    no.adam_step(P, G, m, v, 1, lr=1e-2)
    expect = np.array([1.0, -2.0, 0.5]) - 1e-2 * G["w"] / (np.abs(G["w"]) + 1e-8)
    assert np.allclose(P["w"], expect, rtol=1e-12)


def test_bf16_rounding():
    torch = pytest.importorskip("torch")
    assert no.bf16(1.0) == 1.0
    assert no.bf16(1.0 + 2.0 ** -8) == 1.0                       # tie, to even
    assert no.bf16(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6       # tie, to even
    x = np.random.default_rng(6).standard_normal(1000) * 10.0 ** np.random.default_rng(7).integers(-5, 5, 1000)
    ref = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(no.bf16(x), ref)


def test_trilinear_upsampling():
    x = np.arange(4.0).reshape(1, 4, 1, 1, 1)
    y = no.upsample_trilinear(x, 2)
    # fine centre 0 sits a quarter coarse cell before coarse centre 0 (periodic)
    assert np.isclose(y[0, 0, 0, 0, 0], 0.25 * 3.0 + 0.75 * 0.0)
    assert np.isclose(y[0, 1, 0, 0, 0], 0.75 * 0.0 + 0.25 * 1.0)
    c = np.full((1, 3, 2, 5, 2), 1.5)
    assert np.allclose(no.upsample_trilinear(c, 3), 1.5)
    assert np.allclose(no.upsample_trilinear(x, 1), x)
