"""Python binding of the warm-start network (include/hom_net.h): argument
marshalling only.  Device buffers are torch CUDA tensors; every computation
runs in libhom.so's kernels (no CPU fallback)."""
from __future__ import annotations

import ctypes

import numpy as np

from . import hom as _hom

# every symbol include/hom_net.h declares
EXPORTED = [
    "hom_net_create", "hom_net_destroy", "hom_net_last_error", "hom_net_param_count", "hom_net_get_params",
    "hom_net_set_params", "hom_net_save", "hom_net_load", "hom_net_forward", "hom_net_train_step",
    "hom_net_gradients", "hom_net_warm_start", "hom_net_kernel_launches", "hom_net_conv3d",
    "hom_net_conv3d_wgrad", "hom_net_set_void_weight",
]

# layer names, input and output channels, in parameter order
LAYERS = [("e1a", 1, 16), ("e1b", 16, 16), ("e2a", 16, 32), ("e2b", 32, 32), ("e3a", 32, 48), ("e3b", 48, 48),
          ("bna", 48, 64), ("bnb", 64, 64), ("d3a", 112, 48), ("d3b", 48, 48), ("d2a", 80, 32), ("d2b", 32, 32),
          ("d1a", 48, 16), ("d1b", 16, 16), ("head", 16, 36)]

_ready = False


def load_library():
    global _ready
    lib = _hom.load_library()
    if _ready:
        return lib
    vp, ip, dp, fp = (ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double),
                      ctypes.POINTER(ctypes.c_float))
    lib.hom_net_create.argtypes = [ctypes.POINTER(vp), ctypes.c_ulonglong, vp]
    lib.hom_net_destroy.argtypes = [vp]
    lib.hom_net_destroy.restype = None
    lib.hom_net_last_error.argtypes = []
    lib.hom_net_last_error.restype = ctypes.c_char_p
    lib.hom_net_set_void_weight.argtypes = [vp, ctypes.c_double]
    lib.hom_net_param_count.argtypes = [vp]
    lib.hom_net_param_count.restype = ctypes.c_longlong
    lib.hom_net_get_params.argtypes = [vp, fp]
    lib.hom_net_set_params.argtypes = [vp, fp]
    lib.hom_net_save.argtypes = [vp, ctypes.c_char_p]
    lib.hom_net_load.argtypes = [vp, ctypes.c_char_p]
    lib.hom_net_forward.argtypes = [vp, ctypes.c_int, ip, vp, dp, vp]
    lib.hom_net_train_step.argtypes = [vp, ctypes.c_int, ip, vp, dp, vp, ctypes.c_float, dp]
    lib.hom_net_gradients.argtypes = [vp, ctypes.c_int, ip, vp, dp, vp, fp, dp]
    lib.hom_net_warm_start.argtypes = [vp, ip, ctypes.c_int, vp, ctypes.c_int, dp, vp]
    lib.hom_net_kernel_launches.argtypes = [vp]
    lib.hom_net_kernel_launches.restype = ctypes.c_longlong
    lib.hom_net_conv3d.argtypes = [ctypes.c_int, ip, vp, ctypes.c_int, vp, ctypes.c_int, vp, vp, ctypes.c_int,
                                   ctypes.c_int, vp, ctypes.c_int, vp]
    lib.hom_net_conv3d_wgrad.argtypes = [ctypes.c_int, ip, vp, ctypes.c_int, vp, ctypes.c_int, vp, ctypes.c_int,
                                         vp, vp]
    _ready = True
    return lib


def _check(rc):
    if rc < 0:
        msg = load_library().hom_net_last_error()
        raise _hom.HomError(rc, msg.decode() if msg else "")
    return rc


def _grid(g):
    return (ctypes.c_int * 3)(*[int(v) for v in g])


def _macro(m, count):
    a = np.ascontiguousarray(np.asarray(m, dtype=np.float64).reshape(count, 6))
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


class Net:
    """Owning wrapper of a hom_net*."""

    def __init__(self, seed=0, stream=None):
        lib = load_library()
        h = ctypes.c_void_p()
        _check(lib.hom_net_create(ctypes.byref(h), int(seed), stream))
        self.handle = h

    def close(self):
        if self.handle:
            load_library().hom_net_destroy(self.handle)
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

    def set_void_weight(self, vw):
        _check(load_library().hom_net_set_void_weight(self.handle, float(vw)))

    def param_count(self):
        return int(load_library().hom_net_param_count(self.handle))

    def get_params(self):
        out = np.zeros(self.param_count(), dtype=np.float32)
        _check(load_library().hom_net_get_params(self.handle, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))
        return out

    def set_params(self, flat):
        a = np.ascontiguousarray(flat, dtype=np.float32)
        assert a.size == self.param_count()
        _check(load_library().hom_net_set_params(self.handle, a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))

    def save(self, path):
        _check(load_library().hom_net_save(self.handle, str(path).encode()))

    def load(self, path):
        _check(load_library().hom_net_load(self.handle, str(path).encode()))

    def forward(self, grid, phi, macro, x0):
        """phi [B, V] float32 CUDA tensor, macro [B, 6] (tensor comps), x0 [B, 6, V] output tensor."""
        B = phi.shape[0]
        m, mp = _macro(macro, B)
        _check(load_library().hom_net_forward(self.handle, B, _grid(grid), _hom._ptr(phi), mp, _hom._ptr(x0)))

    def train_step(self, grid, phi, macro, target, lr):
        B = phi.shape[0]
        m, mp = _macro(macro, B)
        loss = ctypes.c_double()
        _check(load_library().hom_net_train_step(self.handle, B, _grid(grid), _hom._ptr(phi), mp, _hom._ptr(target),
                                                 float(lr), ctypes.byref(loss)))
        return loss.value

    def gradients(self, grid, phi, macro, target):
        B = phi.shape[0]
        m, mp = _macro(macro, B)
        g = np.zeros(self.param_count(), dtype=np.float32)
        loss = ctypes.c_double()
        _check(load_library().hom_net_gradients(self.handle, B, _grid(grid), _hom._ptr(phi), mp, _hom._ptr(target),
                                                g.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), ctypes.byref(loss)))
        return g, loss.value

    def warm_start(self, grid, s, phi, macro, x0):
        """phi [V] CUDA tensor on `grid`; the network runs on grid / s; x0 [ncase, 6, V]."""
        m, mp = _macro(macro, int(np.asarray(macro).size // 6))
        _check(load_library().hom_net_warm_start(self.handle, _grid(grid), int(s), _hom._ptr(phi), m.shape[0], mp,
                                                 _hom._ptr(x0)))

    def kernel_launches(self):
        return int(load_library().hom_net_kernel_launches(self.handle))


def unflatten(flat):
    """Flat parameter vector -> {name.W: [27, cout, cin], name.b: [cout]} (float64)."""
    P, o = {}, 0
    for name, ci, co in LAYERS:
        n = 27 * co * ci
        P[name + ".W"] = np.asarray(flat[o:o + n], dtype=np.float64).reshape(27, co, ci)
        o += n
        P[name + ".b"] = np.asarray(flat[o:o + co], dtype=np.float64)
        o += co
    return P


def flatten(P):
    return np.concatenate([np.concatenate([P[n + ".W"].ravel(), P[n + ".b"].ravel()]) for n, _, _ in LAYERS])


def conv3d(grid, src0, W, cout, src1=None, bias=None, relu=False, out=None, stream=None):
    """Step-level convolution on BF16 CUDA tensors (channels-last)."""
    c0s = src0.shape[-1]
    c1s = 0 if src1 is None else src1.shape[-1]
    _check(load_library().hom_net_conv3d(src0.shape[0], _grid(grid), _hom._ptr(src0), c0s,
                                         None if src1 is None else _hom._ptr(src1), c1s, _hom._ptr(W),
                                         None if bias is None else _hom._ptr(bias), int(relu), int(cout),
                                         _hom._ptr(out), 1 if str(out.dtype).endswith("float32") else 0, stream))
    return out


def conv3d_wgrad(grid, G, src0, dW, src1=None, stream=None):
    c0s = src0.shape[-1]
    c1s = 0 if src1 is None else src1.shape[-1]
    _check(load_library().hom_net_conv3d_wgrad(src0.shape[0], _grid(grid), _hom._ptr(G), G.shape[-1],
                                               _hom._ptr(src0), c0s, None if src1 is None else _hom._ptr(src1), c1s,
                                               _hom._ptr(dW), stream))
    return dW
