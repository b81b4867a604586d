"""FP64 CPU oracle of the Galerkin-FFT homogenization method (arXiv 2110.00733).

TEST INFRASTRUCTURE.  This package is the slow, obviously correct reference
that the GPU library is checked against.  Only the tests, the smoke check and
the CPU-baseline leg of the benchmark may import it; the GPU library never
does, and this package never imports the GPU library.

The numerical work is in ``hom_oracle.c`` (plain C, FP64, its own
mixed-radix FFT); this module compiles it with gcc on first use and wraps it
with ctypes.  Fields are 6 x V arrays of Mandel components (section 2.1 stores
the strain at each voxel centre); the wrappers below take and return tensor
components where marked.

Parity pins (tests/test_oracle_*.py): FFT against numpy.fft, the rotated
frequency against its tan form and against the real-space stencil symbol, the
projector's idempotence / Hermitian symmetry / rank, homogeneous and laminate
closed forms, the void laminate, MINRES against SciPy, and a dense real-space
direct solve on odd grids.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hom_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

SQ2 = np.sqrt(2.0)


def build(force: bool = False) -> str:
    """Compile hom_oracle.c into oracle/_build/liboracle.so (gcc, OpenMP)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-std=c11",
           _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = ctypes.CDLL(_LIB)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        lib.orc_fft3d.argtypes = [ip, dp, ctypes.c_int]
        lib.orc_fft1d.argtypes = [ctypes.c_int, dp, ctypes.c_int]
        lib.orc_frequency.argtypes = [ip, ip, ctypes.c_int, dp]
        lib.orc_gamma_apply.argtypes = [dp, dp, dp]
        lib.orc_stiffness_mandel.argtypes = [ctypes.c_double, ctypes.c_double, dp]
        lib.orc_apply.argtypes = [ip, dp, ctypes.c_double, ctypes.c_double,
                                  ctypes.c_int, dp, dp]
        lib.orc_rhs.argtypes = [ip, dp, ctypes.c_double, ctypes.c_double,
                                ctypes.c_int, dp, dp]
        lib.orc_project.argtypes = [ip, ctypes.c_int, dp, dp]
        lib.MATVEC = ctypes.CFUNCTYPE(None, ctypes.c_void_p, dp, dp)
        lib.orc_minres.argtypes = [ctypes.c_long, lib.MATVEC, ctypes.c_void_p,
                                   dp, dp, ctypes.c_double, ctypes.c_int, dp, dp]
        lib.orc_minres.restype = ctypes.c_int
        lib.orc_solve.argtypes = [ip, dp, ctypes.c_double, ctypes.c_double,
                                  ctypes.c_int, dp, ctypes.c_double, ctypes.c_int,
                                  dp, dp, dp, dp]
        lib.orc_solve.restype = ctypes.c_int
        lib.orc_apply_mixed.argtypes = [ip, dp, ctypes.c_double, ctypes.c_double,
                                        ctypes.c_int, ctypes.c_int, dp, dp]
        lib.orc_rhs_mixed.argtypes = [ip, dp, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_int, ctypes.c_int, dp, dp, dp]
        lib.orc_solve_mixed.argtypes = [ip, dp, ctypes.c_double, ctypes.c_double,
                                        ctypes.c_int, ctypes.c_int, dp, dp, ctypes.c_int, ctypes.c_double,
                                        ctypes.c_int, dp, dp, dp, dp, dp]
        lib.orc_cg.argtypes = [ctypes.c_long, lib.MATVEC, ctypes.c_void_p,
                               dp, dp, ctypes.c_double, ctypes.c_int, dp, dp]
        lib.orc_cg.restype = ctypes.c_int
        lib.orc_solve_mixed.restype = ctypes.c_int
        lib.orc_pfs.argtypes = [ip, dp, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double, dp]
        lib.orc_j2_point.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_double, dp, dp, ctypes.c_double, dp, dp, dp, dp]
        lib.orc_j2_increment.argtypes = [ip, dp, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                         ctypes.c_double, ctypes.c_int, ctypes.c_int, dp, dp, dp, dp, dp, dp,
                                         ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_int, dp, dp, dp]
        lib.orc_j2_increment.restype = ctypes.c_int
        lib.orc_num_threads.restype = ctypes.c_int
        lib.orc_modb_apply.argtypes = [ip, dp, ctypes.c_double, ctypes.c_double, ctypes.c_double, dp, dp]
        lib.orc_modb_rhs.argtypes = [ip, dp, ctypes.c_double, ctypes.c_double, dp, dp]
        lib.orc_modb_precond.argtypes = [ip, ctypes.c_double, ctypes.c_double, ctypes.c_double, dp, dp]
        lib.orc_modb_fields.argtypes = [ip, dp, ctypes.c_double, ctypes.c_double, dp, dp, dp, dp]
        _lib = lib
        return lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(seq):
    arr = (ctypes.c_int * len(seq))(*[int(s) for s in seq])
    return arr


def num_threads() -> int:
    return int(_load().orc_num_threads())


# --------------------------------------------------------------------------
# Mandel <-> tensor components (e11, e22, e33, e23, e13, e12)
# --------------------------------------------------------------------------

def tensor_to_mandel(t):
    """(..., 6) or (6, ...) tensor components -> Mandel; axis 0 is the component."""
    m = np.array(t, dtype=np.float64, copy=True)
    m[3:] *= SQ2
    return m


def mandel_to_tensor(m):
    t = np.array(m, dtype=np.float64, copy=True)
    t[3:] /= SQ2
    return t


# --------------------------------------------------------------------------
# Wrapped steps
# --------------------------------------------------------------------------

def fft3d(a: np.ndarray, sign: int = -1) -> np.ndarray:
    """Unnormalised 3-D DFT of a complex array (3-D), sign -1 forward."""
    lib = _load()
    a = np.ascontiguousarray(a, dtype=np.complex128)
    assert a.ndim == 3
    out = a.copy()
    lib.orc_fft3d(_ip(a.shape), out.view(np.float64).ctypes.data_as(
        ctypes.POINTER(ctypes.c_double)), int(sign))
    return out


def fft1d(a: np.ndarray, sign: int = -1) -> np.ndarray:
    lib = _load()
    out = np.ascontiguousarray(a, dtype=np.complex128).copy()
    lib.orc_fft1d(int(out.size), out.view(np.float64).ctypes.data_as(
        ctypes.POINTER(ctypes.c_double)), int(sign))
    return out


def frequency(shape, k, deriv: int) -> np.ndarray:
    """Frequency vector (3 complex) at FFT index k; deriv 0 continuous, 1 rotated."""
    lib = _load()
    out = np.zeros(6)
    lib.orc_frequency(_ip(shape), _ip(k), int(deriv), _dp(out))
    return out[0::2] + 1j * out[1::2]


def gamma_apply(xi, tau_mandel) -> np.ndarray:
    """Projector of eq. (galop) at one frequency on a complex Mandel 6-vector."""
    lib = _load()
    xi = np.asarray(xi, dtype=np.complex128)
    t = np.asarray(tau_mandel, dtype=np.complex128)
    xr = np.ascontiguousarray(np.stack([xi.real, xi.imag], -1).reshape(-1))
    tr = np.ascontiguousarray(np.stack([t.real, t.imag], -1).reshape(-1))
    out = np.zeros(12)
    lib.orc_gamma_apply(_dp(xr), _dp(tr), _dp(out))
    return out[0::2] + 1j * out[1::2]


def stiffness_mandel(E: float, nu: float) -> np.ndarray:
    lib = _load()
    out = np.zeros(36)
    lib.orc_stiffness_mandel(float(E), float(nu), _dp(out))
    return out.reshape(6, 6)


def _phi(phi):
    p = np.ascontiguousarray(phi, dtype=np.float64)
    assert p.ndim == 3
    return p


def apply(phi, E, nu, deriv, eps_mandel) -> np.ndarray:
    """A(eps) of eq. (linearOp); eps, result: (6, N1, N2, N3) Mandel."""
    lib = _load()
    p = _phi(phi)
    e = np.ascontiguousarray(eps_mandel, dtype=np.float64).reshape((6,) + p.shape)
    out = np.empty_like(e)
    lib.orc_apply(_ip(p.shape), _dp(p), float(E), float(nu), int(deriv), _dp(e), _dp(out))
    return out


def rhs(phi, E, nu, deriv, Ebar_tensor) -> np.ndarray:
    """b of eq. (gallin) for a macro strain in tensor components (strain control)."""
    lib = _load()
    p = _phi(phi)
    Eb = np.ascontiguousarray(tensor_to_mandel(np.asarray(Ebar_tensor, dtype=np.float64)))
    out = np.empty((6,) + p.shape)
    lib.orc_rhs(_ip(p.shape), _dp(p), float(E), float(nu), int(deriv), _dp(Eb), _dp(out))
    return out


def project(shape, deriv, field_mandel) -> np.ndarray:
    """F^-1 G F applied to a real 6 x V field (no material)."""
    lib = _load()
    f = np.ascontiguousarray(field_mandel, dtype=np.float64).reshape((6,) + tuple(shape))
    out = np.empty_like(f)
    lib.orc_project(_ip(shape), int(deriv), _dp(f), _dp(out))
    return out


def minres(matvec, b, tol=1e-12, max_it=1000):
    """Oracle MINRES on a Python matvec (used to pin it against SciPy)."""
    lib = _load()
    b = np.ascontiguousarray(b, dtype=np.float64)
    n = b.size
    x = np.zeros(n)
    hist = np.zeros(max_it + 1)
    rel = ctypes.c_double(0.0)

    def cb(_ctx, xp, yp):
        xv = np.ctypeslib.as_array(xp, shape=(n,))
        yv = np.ctypeslib.as_array(yp, shape=(n,))
        yv[:] = matvec(xv.copy())

    cfun = lib.MATVEC(cb)
    it = lib.orc_minres(n, cfun, None, _dp(b), _dp(x), float(tol), int(max_it),
                        ctypes.byref(rel), _dp(hist))
    return x, int(it), float(rel.value), hist[: it + 1]


def solve(phi, E, nu, deriv, Ebar_tensor, tol=1e-10, max_it=5000, history=False):
    """Full Galerkin-MINRES solve for one macro strain (tensor components).

    Returns dict with eps_tilde (6,N1,N2,N3 Mandel), sigma_mean (tensor comps),
    iterations, est_residual, true_residual (eq. galres)."""
    lib = _load()
    p = _phi(phi)
    Eb = np.ascontiguousarray(tensor_to_mandel(np.asarray(Ebar_tensor, dtype=np.float64)))
    eps = np.zeros((6,) + p.shape)
    sig = np.zeros(6)
    info = np.zeros(3)
    hist = np.zeros(max_it + 1)
    lib.orc_solve(_ip(p.shape), _dp(p), float(E), float(nu), int(deriv), _dp(Eb),
                  float(tol), int(max_it), _dp(eps), _dp(sig), _dp(info), _dp(hist))
    it = int(info[0])
    out = {
        "eps_tilde": eps,
        "sigma_mean": mandel_to_tensor(sig),
        "iterations": it,
        "est_residual": float(info[1]),
        "true_residual": float(info[2]),
    }
    if history:
        out["history"] = hist[: it + 1].copy()
    return out


def apply_mixed(phi, E, nu, deriv, mask, eps_mandel) -> np.ndarray:
    """A(eps) with the projector of eq. (galop) for the stress-controlled
    Mandel components in `mask` (bit c = component c of 11, 22, 33, 23, 13, 12)."""
    lib = _load()
    p = _phi(phi)
    e = np.ascontiguousarray(eps_mandel, dtype=np.float64).reshape((6,) + p.shape)
    out = np.empty_like(e)
    lib.orc_apply_mixed(_ip(p.shape), _dp(p), float(E), float(nu), int(deriv), int(mask), _dp(e), _dp(out))
    return out


def rhs_mixed(phi, E, nu, deriv, mask, Ebar_tensor, Sbar_tensor) -> np.ndarray:
    """b of eq. (gallin) under mixed control: strain components outside
    `mask` from Ebar, stress components in `mask` from Sbar (tensor
    components; the other entries of each are ignored)."""
    lib = _load()
    p = _phi(phi)
    Eb = np.ascontiguousarray(tensor_to_mandel(np.asarray(Ebar_tensor, dtype=np.float64)))
    Sb = np.ascontiguousarray(tensor_to_mandel(np.asarray(Sbar_tensor, dtype=np.float64)))
    out = np.empty((6,) + p.shape)
    lib.orc_rhs_mixed(_ip(p.shape), _dp(p), float(E), float(nu), int(deriv), int(mask), _dp(Eb), _dp(Sb),
                      _dp(out))
    return out


def cg(matvec, b, tol=1e-12, max_it=1000):
    """Oracle conjugate gradients on a Python matvec (used to pin it)."""
    lib = _load()
    b = np.ascontiguousarray(b, dtype=np.float64)
    n = b.size
    x = np.zeros(n)
    hist = np.zeros(max_it + 1)
    rel = ctypes.c_double(0.0)

    def cb(_ctx, xp, yp):
        xv = np.ctypeslib.as_array(xp, shape=(n,))
        yv = np.ctypeslib.as_array(yp, shape=(n,))
        yv[:] = matvec(xv.copy())

    cfun = lib.MATVEC(cb)
    it = lib.orc_cg(n, cfun, None, _dp(b), _dp(x), float(tol), int(max_it), ctypes.byref(rel), _dp(hist))
    return x, int(it), float(rel.value), hist[: it + 1]


def solve_mixed(phi, E, nu, deriv, mask, Ebar_tensor, Sbar_tensor, tol=1e-10, max_it=5000, method="minres",
                history=False):
    """Galerkin solve under mixed macroscopic control (eq. galop, eq.
    gallin) by MINRES or CG: Mandel components in `mask` are stress-
    controlled (mean stress Sbar), the others strain-controlled (mean strain
    Ebar), tensor components in and out.

    Returns dict with eps_tilde (6,N1,N2,N3 Mandel, including the mean of the
    stress-controlled components), sigma_mean and eps_mean (tensor comps),
    iterations, est_residual, true_residual."""
    lib = _load()
    p = _phi(phi)
    Eb = np.ascontiguousarray(tensor_to_mandel(np.asarray(Ebar_tensor, dtype=np.float64)))
    Sb = np.ascontiguousarray(tensor_to_mandel(np.asarray(Sbar_tensor, dtype=np.float64)))
    eps = np.zeros((6,) + p.shape)
    sig = np.zeros(6)
    em = np.zeros(6)
    info = np.zeros(3)
    hist = np.zeros(max_it + 1)
    assert method in ("minres", "cg")
    lib.orc_solve_mixed(_ip(p.shape), _dp(p), float(E), float(nu), int(deriv), int(mask), _dp(Eb), _dp(Sb),
                        1 if method == "cg" else 0, float(tol), int(max_it), _dp(eps), _dp(sig), _dp(em),
                        _dp(info), _dp(hist))
    out = {
        "eps_tilde": eps,
        "sigma_mean": mandel_to_tensor(sig),
        "eps_mean": mandel_to_tensor(em),
        "iterations": int(info[0]),
        "est_residual": float(info[1]),
        "true_residual": float(info[2]),
    }
    if history:
        out["history"] = hist[: out["iterations"] + 1].copy()
    return out


def pfs(omega_fine, ratio, ell, eps=1.0, threshold=0.05) -> np.ndarray:
    """Phase-field smoothening (section 3.2, eq. phase3): the indicator
    omega on the fine grid filtered by 1 / (1 + (ell^2/eps) |q|^2) (ell in
    fine voxels), averaged over ratio^3 blocks, values below threshold set
    to 0.  Returns the phase map on the simulation grid."""
    lib = _load()
    w = np.ascontiguousarray(omega_fine, dtype=np.float64)
    assert w.ndim == 3 and all(n % ratio == 0 for n in w.shape)
    out = np.empty(tuple(n // ratio for n in w.shape))
    lib.orc_pfs(_ip(w.shape), _dp(w), int(ratio), float(ell), float(eps), float(threshold), _dp(out))
    return out


def j2_point(E, nu, sy, H, phi, eps_mandel, epsp_mandel, alpha):
    """Radial return of small-strain J2 plasticity with linear isotropic
    hardening for one voxel (stress and consistent tangent times phi),
    Mandel components.  Returns (sigma, tangent 6x6, plastic strain, alpha)."""
    lib = _load()
    e = np.ascontiguousarray(eps_mandel, dtype=np.float64)
    ep = np.ascontiguousarray(epsp_mandel, dtype=np.float64)
    sig, Ct, epn, al = np.zeros(6), np.zeros(36), np.zeros(6), ctypes.c_double(0.0)
    lib.orc_j2_point(float(E), float(nu), float(sy), float(H), float(phi), _dp(e), _dp(ep), float(alpha),
                     _dp(sig), _dp(Ct), _dp(epn), ctypes.byref(al))
    return sig, Ct.reshape(6, 6), epn, al.value


class J2Cell:
    """Elastoplastic cell for the Newton extension (section 2.1.1): total
    strain and plastic strain (6 x V Mandel), hardening variable (V)."""

    def __init__(self, phi, E, nu, sy, H=0.0, deriv=1):
        self.phi = _phi(phi)
        self.E, self.nu, self.sy, self.H, self.deriv = float(E), float(nu), float(sy), float(H), int(deriv)
        shape = (6,) + self.phi.shape
        self.eps = np.zeros(shape)
        self.epsp = np.zeros(shape)
        self.alpha = np.zeros(self.phi.shape)
        self.Ebar = np.zeros(6)             # applied macro strain (tensor components)

    def increment(self, mask, Ebar_tensor, Sbar_tensor, tol_lin=1e-6, tol_newton=5e-3, max_newton=30,
                  max_lin=5000):
        """One load increment to the macro strain Ebar (components outside
        mask) and mean stress Sbar (components in mask), tensor components.
        Returns dict with sigma_mean, eps_mean (tensor), newton and linear
        iterations, r_newton, residual (||b|| / ||b_0|| at exit), accepted."""
        lib = _load()
        Et = np.ascontiguousarray(tensor_to_mandel(self.Ebar))
        En = np.ascontiguousarray(tensor_to_mandel(np.asarray(Ebar_tensor, dtype=np.float64)))
        Sn = np.ascontiguousarray(tensor_to_mandel(np.asarray(Sbar_tensor, dtype=np.float64)))
        sig, em, info = np.zeros(6), np.zeros(6), np.zeros(5)
        lib.orc_j2_increment(_ip(self.phi.shape), _dp(self.phi), self.E, self.nu, self.sy, self.H, self.deriv,
                             int(mask), _dp(self.eps), _dp(self.epsp), _dp(self.alpha), _dp(Et), _dp(En), _dp(Sn),
                             float(tol_lin), float(tol_newton), int(max_newton), int(max_lin), _dp(sig), _dp(em),
                             _dp(info))
        self.Ebar = np.asarray(Ebar_tensor, dtype=np.float64).copy()
        return {"sigma_mean": mandel_to_tensor(sig), "eps_mean": mandel_to_tensor(em),
                "newton": int(info[0]), "linear": int(info[1]), "r_newton": float(info[2]),
                "residual": float(info[3]), "accepted": bool(info[4])}


UNIT_CASES = np.eye(6)  # tensor components; shear cases have e_ab = e_ba = 1


def effective_stiffness(phi, E, nu, deriv, tol=1e-10, max_it=5000):
    """6x6 Voigt effective stiffness from the six unit macro strains.

    Voigt convention sigma = C . (e11, e22, e33, 2e23, 2e13, 2e12); a unit
    shear tensor strain e_ab = 1 is an engineering strain of 2, so those
    columns are the mean stress divided by 2."""
    C = np.zeros((6, 6))
    sols = []
    for J in range(6):
        s = solve(phi, E, nu, deriv, UNIT_CASES[J], tol=tol, max_it=max_it)
        gamma = 1.0 if J < 3 else 2.0
        C[:, J] = s["sigma_mean"] / gamma
        sols.append(s)
    return C, sols


# --------------------------------------------------------------------------
# MoDBFFT (section 2.2): penalised displacement FFT, strain control
# --------------------------------------------------------------------------

def _c(a):
    a = np.ascontiguousarray(a, dtype=np.complex128)
    return a, a.view(np.float64).ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def modb_apply(phi, E, nu, alpha, u_hat) -> np.ndarray:
    """A^alpha(u^) of eq. (modbfftfop); u_hat: (3, N1, N2, N3) full complex spectrum."""
    lib = _load()
    p = _phi(phi)
    u, up = _c(np.asarray(u_hat).reshape((3,) + p.shape))
    out = np.zeros_like(u)
    lib.orc_modb_apply(_ip(p.shape), _dp(p), float(E), float(nu), float(alpha), up,
                       out.view(np.float64).ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return out


def modb_rhs(phi, E, nu, Ebar_tensor) -> np.ndarray:
    """b^alpha of eq. (modbfftfrhs) for a macro strain (tensor comps)."""
    lib = _load()
    p = _phi(phi)
    Eb = np.ascontiguousarray(tensor_to_mandel(np.asarray(Ebar_tensor, dtype=np.float64)))
    out = np.zeros((3,) + p.shape, dtype=np.complex128)
    lib.orc_modb_rhs(_ip(p.shape), _dp(p), float(E), float(nu), _dp(Eb),
                     out.view(np.float64).ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return out


def modb_precond(shape, phibar, E, nu, v) -> np.ndarray:
    """[xi . Cbar . xi]^-1 v of eq. (precf), Cbar = phibar C_m."""
    lib = _load()
    vv, vp = _c(np.asarray(v).reshape((3,) + tuple(shape)))
    out = np.zeros_like(vv)
    lib.orc_modb_precond(_ip(shape), float(phibar), float(E), float(nu), vp,
                         out.view(np.float64).ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return out


def modb_fields(phi, E, nu, Ebar_tensor, u_hat):
    """(fluctuation strain 6xV Mandel, mean stress tensor comps) of a solution."""
    lib = _load()
    p = _phi(phi)
    Eb = np.ascontiguousarray(tensor_to_mandel(np.asarray(Ebar_tensor, dtype=np.float64)))
    u, up = _c(np.asarray(u_hat).reshape((3,) + p.shape))
    eps = np.zeros((6,) + p.shape)
    sig = np.zeros(6)
    lib.orc_modb_fields(_ip(p.shape), _dp(p), float(E), float(nu), _dp(Eb), up, _dp(eps), _dp(sig))
    return eps, mandel_to_tensor(sig)


def modb_solve_dense(phi, E, nu, alpha, Ebar_tensor):
    """Direct solve of the MoDBFFT system on a small grid.  The unknown is a
    real displacement fluctuation (its DFT is Hermitian), so the operator of
    eq. (modbfftfop) is assembled over the real basis of 3 x V displacement
    values: column j is the inverse DFT of A^alpha(DFT(e_j)).  Frequencies
    with xi = 0 carry no equation, which leaves a null space (rigid
    translations and the all-Nyquist modes); the minimum-norm least-squares
    solution removes it.  Returns (u_hat, mean stress tensor comps)."""
    p = _phi(phi)
    shape = p.shape
    V = p.size
    n = 3 * V
    A = np.zeros((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        uh = np.fft.fftn(e.reshape((3,) + shape), axes=(1, 2, 3))
        r = modb_apply(p, E, nu, alpha, uh)
        A[:, j] = np.real(np.fft.ifftn(r, axes=(1, 2, 3))).reshape(-1)
    b = np.real(np.fft.ifftn(modb_rhs(p, E, nu, Ebar_tensor), axes=(1, 2, 3))).reshape(-1)
    u = np.linalg.lstsq(A, b, rcond=1e-12)[0]
    uh = np.fft.fftn(u.reshape((3,) + shape), axes=(1, 2, 3))
    eps, sig = modb_fields(p, E, nu, Ebar_tensor, uh)
    return uh, sig
