"""Python binding of libhom.so (include/hom.h): argument marshalling only.

Every entry point of the C ABI is exposed under the same name.  Buffers may be
numpy arrays (host) or torch CUDA tensors (device; create the context with
``device_ptrs=True``).  All arithmetic runs in the library's CUDA kernels;
there is no CPU fallback, and importing this module on a machine where the
library or a GPU is missing raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "libhom.so")

HOM_OK, HOM_NOT_CONVERGED = 0, 1
HOM_EINVAL, HOM_EUNSUPPORTED_GRID, HOM_ENOMEM, HOM_ECUDA, HOM_ENAN, HOM_ETIMEOUT = -1, -2, -3, -4, -5, -6
HOM_INPUT_PHASE_U8, HOM_INPUT_FRACTION_F32, HOM_INPUT_FRACTION_F64 = 0, 1, 2
HOM_SMOOTH_NONE = 0
HOM_DERIV_CONTINUOUS, HOM_DERIV_ROTATED = 0, 1
HOM_SOLVER_GALERKIN_MINRES, HOM_SOLVER_MODBFFT_CG, HOM_SOLVER_GALERKIN_CG = 0, 1, 2
HOM_PREC_FP32_FIELDS, HOM_PREC_FP64 = 0, 1

# every symbol include/hom.h declares
EXPORTED = [
    "hom_default_options", "hom_create", "hom_solve", "hom_effective_stiffness",
    "hom_fields", "hom_apply", "hom_rhs", "hom_fft_forward", "hom_fft_inverse",
    "hom_project", "hom_apply_spectrum", "hom_time_kernels", "hom_get_info", "hom_kernel_launches", "hom_destroy",
    "hom_last_error", "hom_apply_noalloc", "hom_modb_apply", "hom_modb_rhs", "hom_modb_precond",
    "hom_solve_batch", "hom_autotune", "hom_solve_mixed", "hom_pfs",
    "hom_j2_begin", "hom_j2_increment", "hom_j2_state", "hom_j2_end", "hom_j2_time_kernels",
]


class hom_options(ctypes.Structure):
    _fields_ = [("solver", ctypes.c_int), ("precision", ctypes.c_int),
                ("device_ptrs", ctypes.c_int), ("stream", ctypes.c_void_p),
                ("device", ctypes.c_int), ("refine", ctypes.c_int),
                ("rows3", ctypes.c_int), ("tile2", ctypes.c_int), ("tile1", ctypes.c_int),
                ("staging", ctypes.c_int), ("alpha", ctypes.c_double),
                ("autotune", ctypes.c_int), ("host_loop", ctypes.c_int),
                ("sweep_floor", ctypes.c_double)]


class hom_solve_info(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("status", ctypes.c_int),
                ("sweeps", ctypes.c_int), ("reserved", ctypes.c_int),
                ("est_residual", ctypes.c_double), ("true_residual", ctypes.c_double),
                ("sigma_mean", ctypes.c_double * 6), ("time_ms", ctypes.c_double),
                ("eps_mean", ctypes.c_double * 6)]

    def as_dict(self):
        return {"iterations": self.iterations, "status": self.status, "sweeps": self.sweeps,
                "est_residual": self.est_residual, "true_residual": self.true_residual,
                "sigma_mean": np.array(self.sigma_mean[:]), "time_ms": self.time_ms,
                "eps_mean": np.array(self.eps_mean[:])}


class hom_j2_info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("newton", ctypes.c_int), ("linear", ctypes.c_int),
                ("backtracks", ctypes.c_int), ("r_newton", ctypes.c_double), ("residual", ctypes.c_double),
                ("sigma_mean", ctypes.c_double * 6), ("eps_mean", ctypes.c_double * 6),
                ("time_ms", ctypes.c_double)]

    def as_dict(self):
        return {"status": self.status, "newton": self.newton, "linear": self.linear,
                "backtracks": self.backtracks, "r_newton": self.r_newton, "residual": self.residual,
                "sigma_mean": np.array(self.sigma_mean[:]), "eps_mean": np.array(self.eps_mean[:]),
                "time_ms": self.time_ms, "accepted": self.status == HOM_OK}


class HomError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libhom error {code}: {msg}")
        self.code = code


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libhom.so; raises if it is missing (build with __graft_entry__.build())."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libhom.so not built at {path}; run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    vp, ip, dp = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)
    lib.hom_default_options.argtypes = [ctypes.POINTER(hom_options)]
    lib.hom_default_options.restype = None
    lib.hom_create.argtypes = [ctypes.POINTER(vp), ip, vp, ctypes.c_int, ctypes.c_double,
                               ctypes.c_double, ctypes.c_int, ctypes.c_int,
                               ctypes.POINTER(hom_options)]
    lib.hom_solve.argtypes = [vp, dp, ctypes.c_int, ctypes.c_double, ctypes.c_int, vp,
                              ctypes.POINTER(hom_solve_info)]
    lib.hom_solve_mixed.argtypes = [vp, dp, dp, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int, vp,
                                    ctypes.POINTER(hom_solve_info)]
    lib.hom_pfs.argtypes = [ip, vp, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                            ctypes.c_int, vp]
    lib.hom_j2_begin.argtypes = [vp, ctypes.c_double, ctypes.c_double]
    lib.hom_j2_increment.argtypes = [vp, dp, dp, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                     ctypes.c_int, ctypes.POINTER(hom_j2_info)]
    lib.hom_j2_state.argtypes = [vp, vp, vp, vp]
    lib.hom_j2_end.argtypes = [vp]
    lib.hom_effective_stiffness.argtypes = [vp, dp]
    lib.hom_fields.argtypes = [vp, ctypes.c_int, vp, vp]
    lib.hom_apply.argtypes = [vp, vp, vp]
    lib.hom_rhs.argtypes = [vp, dp, vp]
    lib.hom_fft_forward.argtypes = [vp, vp, vp]
    lib.hom_fft_inverse.argtypes = [vp, vp, vp]
    lib.hom_project.argtypes = [vp, vp, vp]
    lib.hom_apply_spectrum.argtypes = [vp, vp, vp]
    lib.hom_time_kernels.argtypes = [vp, ctypes.c_int, dp, ctypes.c_int]
    lib.hom_j2_time_kernels.argtypes = [vp, ctypes.c_int, dp, ctypes.c_int]
    lib.hom_apply_noalloc.argtypes = [ip, vp, ctypes.c_double, ctypes.c_double, ctypes.c_int, vp, vp, vp]
    lib.hom_modb_apply.argtypes = [vp, vp, vp]
    lib.hom_solve_batch.argtypes = [ctypes.POINTER(vp), ctypes.c_int, dp, ctypes.c_int, ctypes.c_double,
                                    ctypes.c_int, ctypes.POINTER(hom_solve_info)]
    lib.hom_autotune.argtypes = [ip, ctypes.c_int, ip]
    lib.hom_modb_rhs.argtypes = [vp, dp, vp]
    lib.hom_modb_precond.argtypes = [vp, vp, vp]
    lib.hom_get_info.argtypes = [vp, ip, ip, ctypes.POINTER(ctypes.c_longlong)]
    lib.hom_kernel_launches.argtypes = [vp]
    lib.hom_kernel_launches.restype = ctypes.c_longlong
    lib.hom_destroy.argtypes = [vp]
    lib.hom_destroy.restype = None
    lib.hom_last_error.argtypes = [vp]
    lib.hom_last_error.restype = ctypes.c_char_p
    _lib = lib
    return lib


def _ptr(a):
    """Address of a numpy array or torch tensor (contiguous)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.flags.c_contiguous
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        assert a.is_contiguous()
        return a.data_ptr()
    raise TypeError(type(a))


def _check(ctx_handle, rc):
    if rc < 0:
        msg = load_library().hom_last_error(ctx_handle)
        raise HomError(rc, msg.decode() if msg else "")
    return rc


class Context:
    """Owning wrapper of a hom_ctx*; methods call the C entry points."""

    def __init__(self, handle, grid, precision, device_ptrs):
        self.handle = handle
        self.grid = tuple(grid)
        self.V = int(np.prod(grid))
        self.precision = precision
        self.device_ptrs = device_ptrs
        self.dtype = np.float32 if precision == HOM_PREC_FP32_FIELDS else np.float64

    def close(self):
        if self.handle:
            load_library().hom_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def hom_create(grid, phase, input_kind=HOM_INPUT_FRACTION_F32, E=1.0, nu=0.3,
               smoothing=HOM_SMOOTH_NONE, derivative=HOM_DERIV_ROTATED,
               precision=HOM_PREC_FP32_FIELDS, device_ptrs=False, stream=None,
               device=-1, refine=3, shape=(0, 0, 0), staging=0,
               solver=HOM_SOLVER_GALERKIN_MINRES, alpha=0.0, autotune=False,
               sweep_floor=0.0, host_loop=False) -> Context:
    lib = load_library()
    opt = hom_options()
    lib.hom_default_options(ctypes.byref(opt))
    opt.precision = precision
    opt.device_ptrs = 1 if device_ptrs else 0
    opt.stream = stream
    opt.device = device
    opt.refine = refine
    opt.rows3, opt.tile2, opt.tile1 = (int(s) for s in shape)
    opt.staging = int(staging)
    opt.solver = int(solver)
    opt.alpha = float(alpha)
    opt.autotune = 1 if autotune else 0
    opt.sweep_floor = float(sweep_floor)
    opt.host_loop = 1 if host_loop else 0
    h = ctypes.c_void_p()
    g = (ctypes.c_int * 3)(*[int(v) for v in grid])
    rc = lib.hom_create(ctypes.byref(h), g, _ptr(phase), int(input_kind), float(E), float(nu),
                        int(smoothing), int(derivative), ctypes.byref(opt))
    if rc < 0:
        msg = lib.hom_last_error(None)
        raise HomError(rc, msg.decode() if msg else "")
    return Context(h, grid, precision, device_ptrs)


def hom_solve(ctx: Context, macro_strain, tol=1e-6, max_it=1000, warm_start=None):
    """Returns (rc, [info dicts]).  macro_strain: (ncase, 6) tensor components."""
    lib = load_library()
    m = np.ascontiguousarray(np.asarray(macro_strain, dtype=np.float64).reshape(-1, 6))
    ncase = m.shape[0]
    infos = (hom_solve_info * ncase)()
    rc = lib.hom_solve(ctx.handle, m.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ncase,
                       float(tol), int(max_it), _ptr(warm_start), infos)
    _check(ctx.handle, rc)
    return rc, [i.as_dict() for i in infos]


def hom_solve_mixed(ctx: Context, macro_strain, macro_stress, stress_mask, tol=1e-6, max_it=1000,
                    warm_start=None):
    """Mixed macroscopic control: Mandel components whose bit is set in
    stress_mask (bit 0..5 = 11, 22, 33, 23, 13, 12) take their mean stress
    from macro_stress, the others their mean strain from macro_strain (both
    (ncase, 6) tensor components).  Returns (rc, [info dicts]); each info
    carries sigma_mean and eps_mean."""
    lib = load_library()
    m = np.ascontiguousarray(np.asarray(macro_strain, dtype=np.float64).reshape(-1, 6))
    sg = np.ascontiguousarray(np.asarray(macro_stress, dtype=np.float64).reshape(-1, 6))
    assert m.shape == sg.shape
    ncase = m.shape[0]
    infos = (hom_solve_info * ncase)()
    dp = ctypes.POINTER(ctypes.c_double)
    rc = lib.hom_solve_mixed(ctx.handle, m.ctypes.data_as(dp), sg.ctypes.data_as(dp), int(stress_mask), ncase,
                             float(tol), int(max_it), _ptr(warm_start), infos)
    _check(ctx.handle, rc)
    return rc, [i.as_dict() for i in infos]


def hom_pfs(omega_fine, ratio, ell, eps=1.0, threshold=0.05, input_kind=None, out=None):
    """Phase-field smoothening (section 3.2) of the fine-grid phase map
    omega_fine (numpy array, or a CUDA tensor for device pointers) onto the
    grid shape // ratio; ell in fine voxels.  Returns the coarse phase map
    (float64; `out` receives it for CUDA input)."""
    lib = load_library()
    shape = tuple(int(v) for v in omega_fine.shape)
    dev = hasattr(omega_fine, "is_cuda") and omega_fine.is_cuda
    if input_kind is None:
        dt = str(omega_fine.dtype)
        input_kind = (HOM_INPUT_PHASE_U8 if "uint8" in dt else
                      HOM_INPUT_FRACTION_F32 if "float32" in dt else HOM_INPUT_FRACTION_F64)
    coarse = tuple(n // ratio for n in shape)
    if not dev:
        omega_fine = np.ascontiguousarray(omega_fine)
        out = np.empty(coarse, dtype=np.float64)
    assert out is not None, "pass a CUDA float64 output tensor for CUDA input"
    g = (ctypes.c_int * 3)(*shape)
    rc = lib.hom_pfs(g, _ptr(omega_fine), int(input_kind), int(ratio), float(ell), float(eps), float(threshold),
                     1 if dev else 0, _ptr(out))
    if rc < 0:
        msg = lib.hom_last_error(None)
        raise HomError(rc, msg.decode() if msg else "")
    return out


def hom_j2_begin(ctx: Context, yield_stress, hardening=0.0):
    """Zero J2 history (section 2.1.1 / section 5 material) on an FP64
    Galerkin-MINRES context; stresses in the units of E."""
    _check(ctx.handle, load_library().hom_j2_begin(ctx.handle, float(yield_stress), float(hardening)))


def hom_j2_increment(ctx: Context, macro_strain, macro_stress, stress_mask, tol_lin=1e-6, tol_newton=5e-3,
                     max_newton=30, max_lin=5000):
    """One load increment by the damped Newton method; macro_strain and
    macro_stress are 6 tensor components (mean strain of the components not
    in stress_mask, mean stress of those in it).  Returns (rc, info dict)."""
    lib = load_library()
    dp = ctypes.POINTER(ctypes.c_double)
    m = np.ascontiguousarray(np.asarray(macro_strain, dtype=np.float64).reshape(6))
    sg = np.ascontiguousarray(np.asarray(macro_stress, dtype=np.float64).reshape(6))
    info = hom_j2_info()
    rc = lib.hom_j2_increment(ctx.handle, m.ctypes.data_as(dp), sg.ctypes.data_as(dp), int(stress_mask),
                              float(tol_lin), float(tol_newton), int(max_newton), int(max_lin), ctypes.byref(info))
    _check(ctx.handle, rc)
    return rc, info.as_dict()


def hom_j2_state(ctx: Context, strain=None, plastic_strain=None, alpha=None):
    """Total and plastic strain (6 x grid, tensor components) and hardening
    variable (grid) of the history, as float64 arrays (or into the given
    device buffers for device_ptrs contexts)."""
    if not ctx.device_ptrs:
        strain = np.empty((6,) + ctx.grid) if strain is None else strain
        plastic_strain = np.empty((6,) + ctx.grid) if plastic_strain is None else plastic_strain
        alpha = np.empty(ctx.grid) if alpha is None else alpha
    _check(ctx.handle, load_library().hom_j2_state(ctx.handle, _ptr(strain), _ptr(plastic_strain), _ptr(alpha)))
    return strain, plastic_strain, alpha


def hom_j2_end(ctx: Context):
    _check(ctx.handle, load_library().hom_j2_end(ctx.handle))


def hom_effective_stiffness(ctx: Context) -> np.ndarray:
    C = np.zeros(36)
    _check(ctx.handle, load_library().hom_effective_stiffness(
        ctx.handle, C.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
    return C.reshape(6, 6)


def _out(ctx, shape, out):
    if out is not None:
        return out
    assert not ctx.device_ptrs, "pass device output buffers when device_ptrs is set"
    return np.empty(shape, dtype=ctx.dtype)


def hom_fields(ctx: Context, icase: int, strain=None, stress=None, want=("strain", "stress")):
    if strain is None and "strain" in want:
        strain = _out(ctx, (6,) + ctx.grid, None)
    if stress is None and "stress" in want:
        stress = _out(ctx, (6,) + ctx.grid, None)
    _check(ctx.handle, load_library().hom_fields(ctx.handle, int(icase), _ptr(strain), _ptr(stress)))
    return strain, stress


def hom_apply(ctx: Context, eps, out=None):
    out = _out(ctx, (6,) + ctx.grid, out)
    _check(ctx.handle, load_library().hom_apply(ctx.handle, _ptr(eps), _ptr(out)))
    return out


def hom_rhs(ctx: Context, macro_strain, out=None):
    out = _out(ctx, (6,) + ctx.grid, out)
    m = np.ascontiguousarray(macro_strain, dtype=np.float64)
    _check(ctx.handle, load_library().hom_rhs(ctx.handle, m.ctypes.data_as(
        ctypes.POINTER(ctypes.c_double)), _ptr(out)))
    return out


def spectrum_shape(ctx: Context):
    n1, n2, n3 = ctx.grid
    return (n1, n2, n3 // 2 + 1, 6)


def displacement_shape(ctx: Context):
    n1, n2, n3 = ctx.grid
    return (n1, n2, n3 // 2 + 1, 3)


def _cdtype(ctx):
    return np.complex64 if ctx.dtype == np.float32 else np.complex128


def hom_modb_apply(ctx: Context, u, out=None):
    if out is None:
        out = np.empty(displacement_shape(ctx), dtype=_cdtype(ctx))
    _check(ctx.handle, load_library().hom_modb_apply(ctx.handle, _ptr(u), _ptr(out)))
    return out


def hom_modb_rhs(ctx: Context, macro_strain, out=None):
    if out is None:
        out = np.empty(displacement_shape(ctx), dtype=_cdtype(ctx))
    m = np.ascontiguousarray(macro_strain, dtype=np.float64)
    _check(ctx.handle, load_library().hom_modb_rhs(ctx.handle, m.ctypes.data_as(
        ctypes.POINTER(ctypes.c_double)), _ptr(out)))
    return out


def hom_modb_precond(ctx: Context, v, out=None):
    if out is None:
        out = np.empty(displacement_shape(ctx), dtype=_cdtype(ctx))
    _check(ctx.handle, load_library().hom_modb_precond(ctx.handle, _ptr(v), _ptr(out)))
    return out


def hom_fft_forward(ctx: Context, field, spectrum=None):
    if spectrum is None:
        assert not ctx.device_ptrs
        spectrum = np.empty(spectrum_shape(ctx),
                            dtype=np.complex64 if ctx.dtype == np.float32 else np.complex128)
    _check(ctx.handle, load_library().hom_fft_forward(ctx.handle, _ptr(field), _ptr(spectrum)))
    return spectrum


def hom_fft_inverse(ctx: Context, spectrum, field=None):
    field = _out(ctx, (6,) + ctx.grid, field)
    _check(ctx.handle, load_library().hom_fft_inverse(ctx.handle, _ptr(spectrum), _ptr(field)))
    return field


def hom_project(ctx: Context, field, out=None):
    out = _out(ctx, (6,) + ctx.grid, out)
    _check(ctx.handle, load_library().hom_project(ctx.handle, _ptr(field), _ptr(out)))
    return out


def hom_apply_spectrum(ctx: Context, spectrum, out=None):
    """G F C F^-1 G on a spectrum (n1, n2, n3//2+1, 6) complex, Mandel, units of E."""
    if out is None:
        assert not ctx.device_ptrs
        out = np.empty(spectrum_shape(ctx), dtype=np.complex64 if ctx.dtype == np.float32 else np.complex128)
    _check(ctx.handle, load_library().hom_apply_spectrum(ctx.handle, _ptr(spectrum), _ptr(out)))
    return out


# hom_time_kernels order: the launches of one elastic MINRES step
KERNEL_NAMES = ["x2_inv", "x3_c2r_law_energy_r2c", "alpha", "x2_fwd", "x1_fwd_lanczos_inv", "givens"]


def hom_time_kernels(ctx: Context, reps: int = 20) -> dict:
    ms = np.zeros(16)
    n = _check(ctx.handle, load_library().hom_time_kernels(
        ctx.handle, int(reps), ms.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 16))
    return {KERNEL_NAMES[i]: float(ms[i]) for i in range(n)}


J2_KERNEL_NAMES = ["j2_return", "j2_tangent_apply", "x3_c2r_real", "x3_r2c_real"]


def hom_j2_time_kernels(ctx: Context, reps: int = 20) -> dict:
    ms = np.zeros(8)
    n = _check(ctx.handle, load_library().hom_j2_time_kernels(
        ctx.handle, int(reps), ms.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 8))
    return {J2_KERNEL_NAMES[i]: float(ms[i]) for i in range(n)}


def hom_get_info(ctx: Context):
    g = (ctypes.c_int * 3)()
    p = ctypes.c_int()
    w = ctypes.c_longlong()
    _check(ctx.handle, load_library().hom_get_info(ctx.handle, g, ctypes.byref(p), ctypes.byref(w)))
    return tuple(g), p.value, w.value


def hom_kernel_launches(ctx: Context) -> int:
    return int(load_library().hom_kernel_launches(ctx.handle))


def hom_destroy(ctx: Context):
    ctx.close()


def hom_last_error(ctx: Context | None = None) -> str:
    s = load_library().hom_last_error(ctx.handle if ctx else None)
    return s.decode() if s else ""


def hom_apply_noalloc(grid, phi, eps, out, E=1.0, nu=0.3, derivative=HOM_DERIV_ROTATED, stream=None):
    """A(eps) for a small cell without device allocation; phi, eps, out are
    torch CUDA tensors (float32) on the current device.  stream: a raw
    cudaStream_t handle (int, e.g. torch.cuda.Stream().cuda_stream) or None
    for the legacy default stream.  The call only enqueues the work: the
    caller synchronises the stream before reading out."""
    lib = load_library()
    g = (ctypes.c_int * 3)(*[int(v) for v in grid])
    rc = lib.hom_apply_noalloc(g, _ptr(phi), float(E), float(nu), int(derivative), _ptr(eps), _ptr(out),
                               None if stream is None else ctypes.c_void_p(int(stream)))
    _check(None, rc)
    return out


def hom_solve_batch(ctxs, macro_strain, tol=1e-6, max_it=1000):
    """Solve the same macro strains on several cells at once.  Returns
    (rc, [[info per case] per cell])."""
    lib = load_library()
    m = np.ascontiguousarray(np.asarray(macro_strain, dtype=np.float64).reshape(-1, 6))
    ncase, ncell = m.shape[0], len(ctxs)
    handles = (ctypes.c_void_p * ncell)(*[c.handle for c in ctxs])
    infos = (hom_solve_info * (ncase * ncell))()
    rc = lib.hom_solve_batch(handles, ncell, m.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ncase,
                             float(tol), int(max_it), infos)
    _check(None, rc)
    return rc, [[infos[i * ncase + k].as_dict() for k in range(ncase)] for i in range(ncell)]


def hom_autotune(grid, precision=HOM_PREC_FP32_FIELDS):
    lib = load_library()
    g = (ctypes.c_int * 3)(*[int(v) for v in grid])
    out = (ctypes.c_int * 3)()
    _check(None, lib.hom_autotune(g, int(precision), out))
    return tuple(out)
