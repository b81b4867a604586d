"""Pins of the Galerkin projector, eq. (galop), at single frequencies."""
import numpy as np
import pytest

import oracle

SQ2 = np.sqrt(2.0)
MI = [0, 1, 2, 1, 0, 0]
MJ = [0, 1, 2, 2, 2, 1]


def to_tensor(m):
    t = np.zeros((3, 3), dtype=complex)
    for c in range(6):
        v = m[c] if c < 3 else m[c] / SQ2
        t[MI[c], MJ[c]] = v
        t[MJ[c], MI[c]] = v
    return t


def to_mandel(t):
    return np.array([t[MI[c], MJ[c]] * (1 if c < 3 else SQ2) for c in range(6)])


def gamma_matrix(xi):
    cols = [oracle.gamma_apply(xi, e) for e in np.eye(6)]
    return np.array(cols).T


def random_xis(rng, n=20):
    out = []
    for _ in range(n):
        out.append(rng.standard_normal(3) + 1j * rng.standard_normal(3))   # generic complex
        out.append(1j * rng.standard_normal(3))                              # continuous form
    for shape, k in [((8, 8, 8), (1, 2, 3)), ((9, 7, 5), (4, 6, 2)), ((16, 8, 4), (15, 1, 3))]:
        out.append(oracle.frequency(shape, k, 1))
    return out


def test_idempotent_hermitian_rank3():
    rng = np.random.default_rng(1)
    for xi in random_xis(rng):
        G = gamma_matrix(xi)
        assert np.allclose(G @ G, G, atol=1e-12)
        assert np.allclose(G, G.conj().T, atol=1e-12)
        assert abs(np.trace(G) - 3.0) < 1e-12


def test_fixes_compatible_and_kills_orthogonal():
    rng = np.random.default_rng(2)
    for xi in random_xis(rng):
        u = rng.standard_normal(3) + 1j * rng.standard_normal(3)
        comp = 0.5 * (np.outer(u, xi) + np.outer(xi, u))
        m = to_mandel(comp)
        assert np.allclose(oracle.gamma_apply(xi, m), m, atol=1e-11 * np.abs(m).max())
        # a symmetric tau with tau conj(xi) = 0 is projected to zero
        t = to_tensor(rng.standard_normal(6) + 1j * rng.standard_normal(6))
        P = np.eye(3) - np.outer(np.conj(xi), xi) / np.vdot(xi, xi).real  # kills conj(xi)
        t0 = P.T @ t @ P          # t0 conj(xi) = 0 and t0 symmetric
        assert np.allclose(t0 @ np.conj(xi), 0, atol=1e-12)
        assert np.allclose(oracle.gamma_apply(xi, to_mandel(t0)), 0, atol=1e-12)


def test_real_direction_matches_textbook_formula():
    """For xi = i q n (continuous derivative), the projector is the classical
    G_ijkl = 1/2(d_ik n_j n_l + d_il n_j n_k + d_jk n_i n_l + d_jl n_i n_k)
             - n_i n_j n_k n_l."""
    rng = np.random.default_rng(3)
    for _ in range(10):
        n = rng.standard_normal(3)
        n /= np.linalg.norm(n)
        d = np.eye(3)
        G4 = 0.5 * (np.einsum("ik,j,l->ijkl", d, n, n) + np.einsum("il,j,k->ijkl", d, n, n)
                    + np.einsum("jk,i,l->ijkl", d, n, n) + np.einsum("jl,i,k->ijkl", d, n, n)) \
            - np.einsum("i,j,k,l->ijkl", n, n, n, n)
        t = to_tensor(rng.standard_normal(6))
        ref = np.einsum("ijkl,kl->ij", G4, t)
        got = oracle.gamma_apply(1j * 3.7 * n, to_mandel(t))
        assert np.allclose(got, to_mandel(ref), atol=1e-12)


def test_zero_frequency_is_zero():
    assert np.allclose(oracle.gamma_apply(np.zeros(3), np.ones(6)), 0)
