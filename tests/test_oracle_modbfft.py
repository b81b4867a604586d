"""Pins of the oracle's MoDBFFT operator (section 2.2, eqs. modbfftfop,
modbfftfrhs, precf) against closed forms and exact identities."""
import numpy as np
import pytest

import oracle
import rve_inputs as ri
from test_oracle_solver import laminate_closed_form

E_M, NU_M = 110e9, 0.3
ALPHA = 1e-4 * E_M            # section 4.2


def rand_spec(shape, seed):
    """DFT of a random real 3-component field: the displacement spectra the
    operator acts on are those of real fields (Hermitian)."""
    rng = np.random.default_rng(seed)
    return np.fft.fftn(rng.standard_normal((3,) + shape), axes=(1, 2, 3))


def xi_cont(shape, k):
    out = []
    for q in range(3):
        n = shape[q]
        if n % 2 == 0 and 2 * k[q] == n:
            out.append(0.0)
        else:
            m = k[q] if 2 * k[q] < n else k[q] - n
            out.append(1j * 2 * np.pi * m)
    return np.array(out)


def acoustic(xi, lam, mu):
    """(xi . C . xi)_ik for isotropic C: (lam + mu) xi_i xi_k + mu (xi . xi) delta_ik."""
    return (lam + mu) * np.outer(xi, xi) + mu * np.dot(xi, xi) * np.eye(3)


def test_homogeneous_rhs_vanishes():
    phi = np.ones((6, 4, 5))
    scale = E_M * phi.size * 2 * np.pi * 3      # |C E_bar| V max|xi|
    assert np.max(np.abs(oracle.modb_rhs(phi, E_M, NU_M, np.eye(6)[0]))) <= 1e-14 * scale


def test_fully_dense_cell_is_the_acoustic_tensor_and_precond_inverts_it():
    """phi = 1 everywhere: A^(u)(k) = (xi . C_m . xi) u(k), and the
    preconditioner with Cbar = C_m is its exact inverse."""
    shape = (6, 5, 4)
    phi = np.ones(shape)
    u = rand_spec(shape, 1)
    Au = oracle.modb_apply(phi, E_M, NU_M, ALPHA, u)
    lam = E_M * NU_M / ((1 + NU_M) * (1 - 2 * NU_M))
    mu = E_M / (2 * (1 + NU_M))
    for k in [(1, 2, 3), (0, 1, 0), (5, 4, 1), (3, 0, 2)]:
        xi = xi_cont(shape, k)
        ref = acoustic(xi, lam, mu) @ u[(slice(None),) + k]
        if not np.any(xi):
            ref = 0 * ref
        assert np.allclose(Au[(slice(None),) + k], ref, rtol=1e-10, atol=1e-6)
    back = oracle.modb_precond(shape, 1.0, E_M, NU_M, Au)
    live = np.ones(shape, bool)
    for idx in np.ndindex(shape):
        if not np.any(xi_cont(shape, idx)):
            live[idx] = False
    assert np.allclose(back[:, live], u[:, live], rtol=1e-10, atol=1e-10)


def test_empty_cell_is_the_penalty_term_alone():
    """phi = 0 everywhere (chi_v = 1): A^(u)(k) = alpha sym(u (x) xi) . xi."""
    shape = (5, 6, 4)
    phi = np.zeros(shape)
    u = rand_spec(shape, 2)
    Au = oracle.modb_apply(phi, E_M, NU_M, ALPHA, u)
    for k in [(1, 2, 3), (4, 5, 1), (2, 3, 0)]:
        xi = xi_cont(shape, k)
        uu = u[(slice(None),) + k]
        e = 0.5 * (np.outer(uu, xi) + np.outer(xi, uu))
        assert np.allclose(Au[(slice(None),) + k], ALPHA * e @ xi, rtol=1e-10, atol=1e-3)


def test_void_free_operator_is_hermitian():
    """Without empty voxels the operator is -D^H C D: Hermitian."""
    shape = (6, 5, 4)
    phi = ri.random_phi(shape, seed=3, void_fraction=0.0)
    u, v = rand_spec(shape, 4), rand_spec(shape, 5)
    Au = oracle.modb_apply(phi, E_M, NU_M, ALPHA, u)
    Av = oracle.modb_apply(phi, E_M, NU_M, ALPHA, v)
    lhs, rhs = np.vdot(v, Au), np.vdot(Av, u)
    assert abs(lhs - rhs) <= 1e-10 * abs(lhs)


@pytest.mark.parametrize("n1,thick", [(9, (4, 5)), (8, (2, 6))])
def test_laminate_without_voids_matches_closed_form(n1, thick):
    """A layered cell without empty space: the displacement solution with
    continuous frequencies is the exact laminate (no Nyquist content)."""
    vals = [1.0, 0.2]
    phi = ri.laminate((n1, 2, 3), thick, vals, axis=0)
    fr = [t / sum(thick) for t in thick]
    for J in [0, 1, 3, 5]:
        u, sig = oracle.modb_solve_dense(phi, E_M, NU_M, ALPHA, np.eye(6)[J])
        ref = laminate_closed_form(vals, fr, np.eye(6)[J])
        assert np.allclose(sig, ref, rtol=1e-9, atol=1e-9 * E_M), (J, sig, ref)
