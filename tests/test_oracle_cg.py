"""Pins of the oracle's conjugate gradients (the solver the paper names for
the Galerkin system of a cell without void, section 2.1) by properties that
hold for CG in exact arithmetic, and against the pinned MINRES on the
Galerkin system of a cell without void."""
import numpy as np
import pytest

import oracle
import rve_inputs as ri

E_M, NU_M = 110e9, 0.3


def spd(n, eigs, seed, basis=False):
    q, _ = np.linalg.qr(np.random.default_rng(seed).standard_normal((n, n)))
    A = (q * eigs) @ q.T
    return (A, q) if basis else A


def test_cg_converges_in_as_many_steps_as_distinct_eigenvalues():
    """With m distinct eigenvalues the Krylov space holds the solution after
    m steps."""
    n = 40
    eigs = np.repeat([1.0, 2.5, 7.0, 30.0, 100.0], 8)
    A = spd(n, eigs, 0)
    b = np.random.default_rng(1).standard_normal(n)
    x, it, rel, _ = oracle.cg(lambda v: A @ v, b, tol=1e-11, max_it=40)
    assert it <= 6
    assert np.allclose(x, np.linalg.solve(A, b), rtol=0, atol=1e-9 * np.linalg.norm(np.linalg.solve(A, b)))


def test_cg_error_in_the_energy_norm_never_grows():
    """x_k minimises the A-norm error over the k-th Krylov space, so the
    error after k steps is non-increasing in k."""
    n = 30
    A = spd(n, np.geomspace(1.0, 1e3, n), 2)
    b = np.random.default_rng(3).standard_normal(n)
    xs = np.linalg.solve(A, b)
    errs = []
    for k in range(1, 25):
        x, it, _, _ = oracle.cg(lambda v: A @ v, b, tol=0.0, max_it=k)
        assert it == k
        d = x - xs
        errs.append(float(d @ A @ d))
    assert all(b2 <= b1 * (1 + 1e-10) for b1, b2 in zip(errs, errs[1:]))
    assert errs[-1] < 1e-2 * errs[0]


def test_cg_on_a_consistent_singular_system_stays_in_the_range():
    """b in the range of a positive semidefinite A: from x0 = 0 every iterate
    lies in the range, and CG reaches the minimum-norm solution."""
    n = 30
    eigs = np.concatenate([np.zeros(5), np.linspace(1.0, 50.0, n - 5)])
    A, q = spd(n, eigs, 4, basis=True)
    y = np.random.default_rng(5).standard_normal(n)
    b = A @ y
    x, it, rel, _ = oracle.cg(lambda v: A @ v, b, tol=1e-12, max_it=200)
    assert rel <= 1e-12
    qr = q[:, 5:]                       # the range of A
    xmin = qr @ (qr.T @ y)              # minimum-norm solution: y projected on the range
    assert np.allclose(x, xmin, rtol=0, atol=1e-9 * np.linalg.norm(xmin))


@pytest.mark.parametrize("deriv", [0, 1])
def test_galerkin_cg_equals_minres_without_void(deriv):
    """phi in [0.05, 1]: the Galerkin system is definite on compatible fields
    and CG converges to the MINRES solution."""
    phi, _ = ri.octet(12, 0.2)
    phi = 0.05 + 0.95 * phi
    Eb = np.array([1e-3, -2e-4, 0, 3e-4, 0, 0])
    a = oracle.solve_mixed(phi, E_M, NU_M, deriv, 0, Eb, np.zeros(6), tol=1e-11, max_it=2000, method="minres")
    b = oracle.solve_mixed(phi, E_M, NU_M, deriv, 0, Eb, np.zeros(6), tol=1e-11, max_it=2000, method="cg")
    assert b["true_residual"] <= 1e-10
    assert np.allclose(b["sigma_mean"], a["sigma_mean"], rtol=1e-9, atol=1e-9 * np.max(np.abs(a["sigma_mean"])))
    assert np.allclose(b["eps_tilde"], a["eps_tilde"], rtol=0, atol=1e-8 * np.max(np.abs(a["eps_tilde"])))
