"""Pins of the oracle's operator, MINRES and effective stiffness against
closed forms, SciPy and a dense real-space direct solve."""
import itertools

import numpy as np
import pytest

import oracle
import rve_inputs as ri

SQ2 = np.sqrt(2.0)
E_M, NU_M = 110e9, 0.3


def voigt_from_mandel_cols(sig_cases):
    """sig_cases[J] = mean stress (tensor comps) for unit tensor strain J."""
    C = np.zeros((6, 6))
    for J, s in enumerate(sig_cases):
        C[:, J] = s / (1.0 if J < 3 else 2.0)
    return C


def voigt_stiffness(E, nu):
    lam = E * nu / ((1 + nu) * (1 - 2 * nu))
    mu = E / (2 * (1 + nu))
    C = np.zeros((6, 6))
    C[:3, :3] = lam
    C[np.arange(3), np.arange(3)] += 2 * mu
    C[np.arange(3, 6), np.arange(3, 6)] = mu
    return C


# ---------------------------------------------------------------- homogeneous
@pytest.mark.parametrize("deriv", [0, 1])
def test_homogeneous_cell_gives_scaled_stiffness(deriv):
    """phi = c everywhere: b = 0, eps_tilde = 0, C_eff = c C_m exactly (b is
    zero up to FFT round-off, so the fluctuation is round-off sized)."""
    phi = np.full((6, 5, 4), 0.37)
    for J in range(6):
        b = oracle.rhs(phi, E_M, NU_M, deriv, np.eye(6)[J])
        assert np.max(np.abs(b)) <= 1e-6 * E_M * 1e-9
    C, sols = oracle.effective_stiffness(phi, E_M, NU_M, deriv)
    assert all(np.max(np.abs(s["eps_tilde"])) <= 1e-14 for s in sols)
    assert np.allclose(C, 0.37 * voigt_stiffness(E_M, NU_M), rtol=1e-13)


# ------------------------------------------------------------------ laminates
def laminate_closed_form(phis, fracs, Ebar_t, E=E_M, nu=NU_M):
    """Layers normal to e1: eps_r = Ebar + sym(a_r x e1), equal traction
    sigma_r . e1, sum_r f_r a_r = 0.  Mandel algebra, independent of FFTs."""
    Cm = np.zeros((6, 6))
    lam = E * nu / ((1 + nu) * (1 - 2 * nu))
    mu = E / (2 * (1 + nu))
    Cm[:3, :3] = lam
    Cm += 2 * mu * np.eye(6)
    B = np.zeros((6, 3))          # sym(a x e1) in Mandel = B a
    B[0, 0] = 1.0
    B[5, 1] = 1.0 / SQ2
    B[4, 2] = 1.0 / SQ2
    Em = np.array(Ebar_t, float)
    Em[3:] *= SQ2
    Ks = [B.T @ (p * Cm) @ B for p in phis]
    Kinv = [np.linalg.inv(K) for K in Ks]
    lhs = sum(f * Ki for f, Ki in zip(fracs, Kinv))
    rhs = sum(f * Ki @ B.T @ (p * Cm) @ Em for f, Ki, p in zip(fracs, Kinv, phis))
    t = np.linalg.solve(lhs, rhs)
    sig = np.zeros(6)
    for f, Ki, p in zip(fracs, Kinv, phis):
        a = Ki @ (t - B.T @ (p * Cm) @ Em)
        sig += f * (p * Cm) @ (Em + B @ a)
    sig[3:] /= SQ2
    return sig


@pytest.mark.parametrize("deriv", [0, 1])
@pytest.mark.parametrize("n1,thick", [(9, (4, 5)), (8, (2, 6)), (12, (4, 2, 6))])
def test_laminate_matches_closed_form(deriv, n1, thick):
    """Odd N, or even N with even layer thicknesses: the pattern has no
    Nyquist component and the discrete solution is the exact laminate one."""
    vals = [1.0, 0.2, 0.55][: len(thick)]
    phi = ri.laminate((n1, 3, 4), thick, vals, axis=0)
    fr = [t / sum(thick) for t in thick]
    for J in range(6):
        Eb = np.eye(6)[J]
        s = oracle.solve(phi, E_M, NU_M, deriv, Eb, tol=1e-13, max_it=500)
        ref = laminate_closed_form(vals, fr, Eb)
        assert np.allclose(s["sigma_mean"], ref, rtol=1e-9, atol=1e-9 * E_M), (J, s["sigma_mean"], ref)


@pytest.mark.parametrize("deriv", [0, 1])
def test_void_laminate_is_plane_stress(deriv):
    """Plates (phi=1) separated by empty layers (phi=0): the traction on the
    plate faces vanishes, so the in-plane block of C_eff is f times the
    plane-stress stiffness and every entry touching e1 is zero.  This is the
    singular case of section 2.1 (zero-stiffness phase)."""
    phi = ri.laminate((10, 4, 4), (4, 6), (1.0, 0.0), axis=0)
    f = 0.4
    sig = []
    for J in range(6):
        s = oracle.solve(phi, E_M, NU_M, deriv, np.eye(6)[J], tol=1e-13, max_it=500)
        assert s["true_residual"] < 1e-10
        sig.append(s["sigma_mean"])
    C = voigt_from_mandel_cols(sig)
    E, nu = E_M, NU_M
    Q = E / (1 - nu ** 2)
    ref = np.zeros((6, 6))
    ref[1, 1] = ref[2, 2] = f * Q
    ref[1, 2] = ref[2, 1] = f * Q * nu
    ref[3, 3] = f * E / (2 * (1 + nu))   # in-plane shear 23
    assert np.allclose(C, ref, atol=1e-9 * E_M)


# --------------------------------------------------------------------- MINRES
def test_minres_matches_scipy_on_singular_consistent_systems():
    scipy_minres = pytest.importorskip("scipy.sparse.linalg").minres
    rng = np.random.default_rng(5)
    for trial in range(4):
        n = 40
        Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
        lam = rng.uniform(-3, 5, n)
        lam[rng.choice(n, 8, replace=False)] = 0.0        # singular
        A = Q @ np.diag(lam) @ Q.T
        b = A @ rng.standard_normal(n)                     # consistent
        x, it, rel, hist = oracle.minres(lambda v: A @ v, b, tol=1e-13, max_it=400)
        xs, info = scipy_minres(A, b, rtol=1e-13, maxiter=400)
        assert np.linalg.norm(A @ x - b) <= 1e-10 * np.linalg.norm(b)
        # both start at 0 and stay in range(A): the minimum-norm solution
        xmin = np.linalg.pinv(A, rcond=1e-10) @ b
        assert np.allclose(x, xmin, atol=1e-8 * np.linalg.norm(xmin))
        assert np.allclose(x, xs, atol=1e-7 * np.linalg.norm(xmin))
        # estimated residual history is monotone non-increasing
        assert np.all(np.diff(hist) <= 1e-14)


# ------------------------------------------------------- dense direct (N odd)
def dense_real_space_solution(phi, Ebar_t, E=E_M, nu=NU_M):
    """Energy minimisation over nodal displacements with the rotated-stencil
    strain (forward difference averaged over the four parallel voxel edges),
    solved by a minimum-norm least-squares dense solve."""
    shape = phi.shape
    V = phi.size
    idx = np.arange(V).reshape(shape)
    Cm = oracle.stiffness_mandel(E, nu)
    # D: (6V) x (3V), Mandel strain of nodal displacement u[i*V + node]
    Dgrad = np.zeros((3, 3, V, V))     # d u_i / d x_p at voxel <- u_i at node
    for p in range(3):
        others = [r for r in range(3) if r != p]
        for c in itertools.product([0, 1], repeat=2):
            sh = [0, 0, 0]
            for r, cr in zip(others, c):
                sh[r] = cr
            n0 = np.roll(idx, [-s for s in sh], axis=(0, 1, 2))
            n1 = np.roll(n0, -1, axis=p)
            for v in range(V):
                vv = np.unravel_index(v, shape)
                Dgrad[p, p, v, n1[vv]] += shape[p] / 4.0   # placeholder axis i = p (filled below)
                Dgrad[p, p, v, n0[vv]] -= shape[p] / 4.0
    G = Dgrad[np.arange(3), np.arange(3)]   # (3 axes p, V, V): derivative operator along p
    D = np.zeros((6 * V, 3 * V))
    MI = [0, 1, 2, 1, 0, 0]
    MJ = [0, 1, 2, 2, 2, 1]
    for c in range(6):
        i, j = MI[c], MJ[c]
        w = 1.0 if c < 3 else SQ2
        # eps_ij = 1/2 (d_j u_i + d_i u_j)
        D[c * V:(c + 1) * V, i * V:(i + 1) * V] += 0.5 * w * G[j]
        D[c * V:(c + 1) * V, j * V:(j + 1) * V] += 0.5 * w * G[i]
    Cbig = np.kron(Cm, np.diag(phi.reshape(-1)))
    Em = np.array(Ebar_t, float)
    Em[3:] *= SQ2
    Ebig = np.repeat(Em, V)
    K = D.T @ Cbig @ D
    f = -D.T @ Cbig @ Ebig
    u = np.linalg.lstsq(K, f, rcond=1e-12)[0]
    eps = D @ u
    sig = Cbig @ (Ebig + eps)
    return eps.reshape((6,) + shape), sig.reshape(6, V).mean(axis=1)


@pytest.mark.parametrize("shape,seed", [((5, 5, 5), 0), ((3, 5, 7), 1)])
def test_dense_direct_solve_odd_grid(shape, seed):
    phi = ri.random_phi(shape, seed=seed, void_fraction=0.35)
    for J in [0, 3, 5]:
        Eb = np.eye(6)[J]
        eps_d, sig_d = dense_real_space_solution(phi, Eb)
        s = oracle.solve(phi, E_M, NU_M, 1, Eb, tol=1e-13, max_it=3000)
        sig_o = oracle.tensor_to_mandel(s["sigma_mean"])
        assert np.allclose(sig_o, sig_d, rtol=1e-8, atol=1e-8 * E_M)
        solid = phi > 0
        diff = (s["eps_tilde"] - eps_d)[:, solid]
        assert np.linalg.norm(diff) <= 1e-7 * np.linalg.norm(eps_d[:, solid])


# --------------------------------------------------------- operator symmetry
@pytest.mark.parametrize("deriv", [0, 1])
def test_operator_symmetric_on_compatible_fields(deriv):
    shape = (6, 5, 7)
    phi = ri.random_phi(shape, seed=3)
    x = oracle.project(shape, deriv, ri.random_field(shape, 1))
    y = oracle.project(shape, deriv, ri.random_field(shape, 2))
    Ax = oracle.apply(phi, 1.0, NU_M, deriv, x)
    Ay = oracle.apply(phi, 1.0, NU_M, deriv, y)
    assert abs(np.vdot(y, Ax) - np.vdot(Ay, x)) <= 1e-12 * np.linalg.norm(Ax) * np.linalg.norm(y)
    assert np.vdot(x, Ax) >= -1e-12     # semidefinite
    # projection is idempotent on fields
    assert np.allclose(oracle.project(shape, deriv, x), x, atol=1e-12)


# ---------------------------------------------------------- octet cell checks
@pytest.fixture(scope="module")
def octet_ceff():
    phi, r = ri.octet(12, 0.15)
    C, sols = oracle.effective_stiffness(phi, E_M, NU_M, 1, tol=1e-10, max_it=3000)
    return phi, C, sols


def test_octet_symmetries_and_voigt_bound(octet_ceff):
    phi, C, sols = octet_ceff
    nrm = np.linalg.norm(C)
    assert np.allclose(C, C.T, atol=1e-7 * nrm)                       # major symmetry
    for a, b in [(0, 1), (1, 2)]:
        assert abs(C[a, a] - C[b, b]) <= 1e-7 * nrm                   # cubic
    assert abs(C[0, 1] - C[0, 2]) <= 1e-7 * nrm and abs(C[0, 1] - C[1, 2]) <= 1e-7 * nrm
    assert abs(C[3, 3] - C[4, 4]) <= 1e-7 * nrm and abs(C[3, 3] - C[5, 5]) <= 1e-7 * nrm
    off = C.copy()
    off[:3, :3] = 0
    off[np.arange(3, 6), np.arange(3, 6)] = 0
    assert np.max(np.abs(off)) <= 1e-7 * nrm
    # Voigt bound <phi> C_m - C_eff is positive semidefinite (Mandel form)
    W = np.diag([1, 1, 1, SQ2, SQ2, SQ2])
    Cv = W @ (phi.mean() * voigt_stiffness(E_M, NU_M) - C) @ W
    assert np.min(np.linalg.eigvalsh(0.5 * (Cv + Cv.T))) >= -1e-7 * nrm
    for s in sols:
        assert s["true_residual"] < 1e-8


def test_linearity_in_macro_strain(octet_ceff):
    phi = octet_ceff[0]
    e1, e2 = np.eye(6)[0], np.eye(6)[4]
    s1 = oracle.solve(phi, E_M, NU_M, 1, e1, tol=1e-11)
    s2 = oracle.solve(phi, E_M, NU_M, 1, e2, tol=1e-11)
    s12 = oracle.solve(phi, E_M, NU_M, 1, 2.0 * e1 - 0.5 * e2, tol=1e-11)
    lin = 2.0 * s1["sigma_mean"] - 0.5 * s2["sigma_mean"]
    assert np.allclose(s12["sigma_mean"], lin, rtol=1e-8, atol=1e-8 * E_M)
