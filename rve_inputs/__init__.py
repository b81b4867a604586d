"""Seeded synthetic inputs for the homogenization solver.

This module generates phase maps (per-voxel solid fraction phi) and macro
strains.  It holds geometry and random-number generation only -- none of the
homogenization arithmetic -- and it is the one module that both the CPU
oracle's tests and the GPU library's tests and benchmark draw inputs from.

* ``octet(n, rho, ...)``: octet-truss cell (FCC nearest-neighbour struts,
  periodic capsules), phi from s^3 sub-voxel sampling (Voigt fine grid,
  section 3.3), strut radius solved so that mean(phi) = rho (section 4.3).
* ``laminate(n, ...)``: layered phase map normal to x1 (closed-form pins).
* ``random_phi(n, ...)``: i.i.d. phases for operator parity tests.
* ``unit_sphere_strain(rng)``: macro strain uniform on the Mandel unit sphere.
* ``as_printed(n, ...)``: a synthetic stand-in for the scanned as-printed cell
  of section 6: octet cells whose strut surface is moved by a Gaussian random
  field, with random spherical pores.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "voxelize.c")
_LIB = os.path.join(_HERE, "_build", "libvoxelize.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    subprocess.run(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-std=c11",
                    _SRC, "-o", tmp, "-lm"], check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            fp = ctypes.POINTER(ctypes.c_float)
            ip = ctypes.POINTER(ctypes.c_int)
            lib.octet_phi.argtypes = [fp, ip, ctypes.c_int, ctypes.c_double,
                                      ctypes.c_int, fp]
            lib.octet_phi.restype = ctypes.c_double
            lib.octet_center_distance.argtypes = [fp, ip, ctypes.c_int]
            lib.octet_phi_at_radius.argtypes = [fp, ip, ctypes.c_int, ctypes.c_double, ctypes.c_int, fp]
            lib.octet_subpoint_distances.argtypes = [fp, ip, ctypes.c_int, ctypes.c_int]
            _lib = lib
    return _lib


def _grid(n):
    if np.isscalar(n):
        return (int(n),) * 3
    g = tuple(int(v) for v in n)
    assert len(g) == 3
    return g


def octet(n, rho: float, sub: int = 4, cells: int = 1, dist_perturb=None):
    """Octet-truss phase map on an n^3 (or n1 x n2 x n3) grid.

    Returns (phi float32 array of shape (n1,n2,n3), strut radius in
    unit-cell lengths)."""
    lib = _load()
    g = _grid(n)
    phi = np.zeros(g, dtype=np.float32)
    pert = None
    if dist_perturb is not None:
        pert = np.ascontiguousarray(dist_perturb, dtype=np.float32).reshape(g)
    r = lib.octet_phi(phi.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                      (ctypes.c_int * 3)(*g), int(cells), float(rho), int(sub),
                      None if pert is None else pert.ctypes.data_as(ctypes.POINTER(ctypes.c_float)))
    if r < 0:
        raise RuntimeError("octet voxelizer could not bracket the strut radius")
    return phi, float(r)


def octet_at_radius(n, r: float, sub: int = 4, cells: int = 1, dist_perturb=None):
    """phi for a given strut radius, every voxel sub-sampled (slow; tests)."""
    lib = _load()
    g = _grid(n)
    phi = np.zeros(g, dtype=np.float32)
    pert = None
    if dist_perturb is not None:
        pert = np.ascontiguousarray(dist_perturb, dtype=np.float32).reshape(g)
    fp = ctypes.POINTER(ctypes.c_float)
    lib.octet_phi_at_radius(phi.ctypes.data_as(fp), (ctypes.c_int * 3)(*g), int(cells), float(r), int(sub),
                            None if pert is None else pert.ctypes.data_as(fp))
    return phi


class OctetFamily:
    """Octet cells of one grid at many densities: the sub-sample distances are
    computed once; a density is then a radius (the matching quantile of all
    sub-sample distances, midway between neighbours; where equal distances
    make the exact count unreachable, the nearer end of the run of ties, as
    octet() does) and a threshold."""

    def __init__(self, n, sub: int = 4, cells: int = 1):
        lib = _load()
        self.grid = _grid(n)
        self.S = sub ** 3
        V = int(np.prod(self.grid))
        d = np.zeros(V * self.S, dtype=np.float32)
        lib.octet_subpoint_distances(d.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                     (ctypes.c_int * 3)(*self.grid), int(cells), int(sub))
        self.d = d.reshape(V, self.S)
        self.sorted = np.sort(d)

    def radius(self, rho: float) -> float:
        sd = self.sorted
        k = int(round(rho * sd.size))
        k = min(max(k, 1), sd.size - 1)
        a = int(np.searchsorted(sd, sd[k - 1], side="left"))     # first of the ties
        b = int(np.searchsorted(sd, sd[k - 1], side="right"))    # past the ties
        cnt = a if k - a <= b - k else b
        if cnt < 1:
            cnt = b
        if cnt >= sd.size:
            cnt = a
        return 0.5 * (float(sd[cnt - 1]) + float(sd[cnt]))

    def phi(self, rho: float):
        r = np.float32(self.radius(rho))
        return ((self.d < r).sum(axis=1, dtype=np.int32).astype(np.float32) / self.S).reshape(self.grid)


def va_phase(signed_distance, voxel: float):
    """Voigt analytic phase map (section 3.3, eq. phaselin): 1 where the voxel
    centre lies deeper than half a voxel inside the material, 0 deeper than
    half a voxel outside, and in between linear in the signed distance D of
    the centre to the surface (positive in the material), phi = 1/2 + D / l
    with l the voxel length: the exact volume fraction for a planar surface."""
    return np.clip(0.5 + np.asarray(signed_distance, dtype=np.float64) / voxel, 0.0, 1.0)


def octet_va(n: int, rho: float, cells: int = 1):
    """Octet phase map by Voigt analytic smoothening, with the strut radius of
    octet(n, rho) (whose map sub-samples each voxel, the paper's fine-grid
    Voigt rule): returns (phi float32 (n, n, n), radius).  Cubic grids only."""
    _, r = octet(n, rho, cells=cells)
    d = octet_center_distance(n, cells).astype(np.float64)
    return va_phase(r - d, cells / n).astype(np.float32), r


def octet_center_distance(n, cells: int = 1):
    lib = _load()
    g = _grid(n)
    out = np.zeros(g, dtype=np.float32)
    lib.octet_center_distance(out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                              (ctypes.c_int * 3)(*g), int(cells))
    return out


def laminate(n, thickness, values, axis: int = 0):
    """Layered phase map: consecutive layers of the given thicknesses (voxels)
    along `axis`, taking the given phi values, repeated to fill the grid."""
    g = _grid(n)
    pattern = np.concatenate([np.full(t, v, dtype=np.float64)
                              for t, v in zip(thickness, values)])
    assert g[axis] % pattern.size == 0, "layers must tile the axis"
    line = np.tile(pattern, g[axis] // pattern.size)
    shape = [1, 1, 1]
    shape[axis] = g[axis]
    return np.broadcast_to(line.reshape(shape), g).astype(np.float64).copy()


def random_phi(n, seed: int, void_fraction: float = 0.3, fractional: bool = True):
    """i.i.d. phase map: a `void_fraction` of voxels empty (phi = 0), the rest
    uniform in (0.05, 1] (or exactly 1 when fractional is False)."""
    g = _grid(n)
    rng = np.random.default_rng(seed)
    phi = rng.uniform(0.05, 1.0, size=g) if fractional else np.ones(g)
    phi[rng.random(g) < void_fraction] = 0.0
    return phi


def random_field(n, seed: int, ncomp: int = 6):
    """Seeded standard-normal field of shape (ncomp, n1, n2, n3)."""
    g = _grid(n)
    return np.random.default_rng(seed).standard_normal((ncomp,) + g)


def unit_sphere_strain(rng) -> np.ndarray:
    """Macro strain, tensor components (e11,e22,e33,e23,e13,e12), drawn
    uniformly on the unit sphere of the Mandel norm."""
    m = rng.standard_normal(6)
    m /= np.linalg.norm(m)
    t = m.copy()
    t[3:] /= np.sqrt(2.0)
    return t


def gaussian_random_field(n, seed: int, corr_len: float = 3.0, std: float = 1.0):
    """Periodic Gaussian random field on an n^3 grid (voxel units): seeded
    white noise filtered by exp(-|k|^2 l^2 / 4), i.e. covariance
    exp(-d^2 / (2 l^2)) up to normalisation, rescaled to the given standard
    deviation."""
    g = _grid(n)
    rng = np.random.default_rng(seed)
    w = rng.standard_normal(g).astype(np.float32)
    k = [np.fft.fftfreq(m) * 2 * np.pi for m in g]
    kz = np.fft.rfftfreq(g[2]) * 2 * np.pi
    k2 = k[0][:, None, None] ** 2 + k[1][None, :, None] ** 2 + kz[None, None, :] ** 2
    filt = np.exp(-k2 * corr_len ** 2 / 4.0).astype(np.float32)
    f = np.fft.irfftn(np.fft.rfftn(w) * filt, s=g, axes=(0, 1, 2)).astype(np.float32)
    f -= f.mean()
    f *= std / f.std()
    return f


def add_pores(phi, seed: int, porosity: float = 0.01, rmin: float = 2.0, rmax: float = 8.0):
    """Carve spheres of radius U[rmin, rmax] voxels, centres drawn uniformly
    and kept only inside the solid (phi >= 0.5), until the removed solid
    volume reaches `porosity` of the solid volume.  Periodic.  In place."""
    rng = np.random.default_rng(seed)
    g = phi.shape
    target = porosity * float(phi.sum(dtype=np.float64))
    removed = 0.0
    tries = 0
    while removed < target and tries < 1000000:
        tries += 1
        c = [int(rng.integers(0, m)) for m in g]
        if phi[c[0], c[1], c[2]] < 0.5:
            continue
        r = rng.uniform(rmin, rmax)
        R = int(np.ceil(r))
        idx = [np.arange(c[a] - R, c[a] + R + 1) % g[a] for a in range(3)]
        d = [np.arange(-R, R + 1, dtype=np.float32) ** 2 for _ in range(3)]
        inside = (d[0][:, None, None] + d[1][None, :, None] + d[2][None, None, :]) <= r * r
        block = phi[np.ix_(idx[0], idx[1], idx[2])]
        removed += float(block[inside].sum(dtype=np.float64))
        block[inside] = 0.0
        phi[np.ix_(idx[0], idx[1], idx[2])] = block
    return phi


def as_printed(n: int = 512, cells: int = 2, rho: float = 0.12, seed: int = 0, corr_len: float = 3.0,
               std: float = 1.0, porosity: float = 0.01):
    """Synthetic as-printed lattice: `cells`^3 octet cells on an n^3 grid whose
    strut surface moves by a Gaussian random field (correlation length
    `corr_len`, standard deviation `std`, both in voxels; interpolated
    trilinearly to the sub-sample points and added to the axis distance),
    Voigt fractions from 4^3 sub-samples at the target density, then
    spherical pores removing `porosity` of the solid.  Returns
    (phi float32, radius)."""
    g = _grid(n)
    grf = gaussian_random_field(g, seed, corr_len, std)
    # a distance perturbation of one voxel is cells / n unit-cell lengths
    phi, r = octet(g, rho, sub=4, cells=cells, dist_perturb=grf * (cells / g[0]))
    add_pores(phi, seed + 1, porosity)
    return phi, r
