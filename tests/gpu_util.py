"""Shared helpers of the GPU parity tests (no method arithmetic here)."""
import numpy as np

FP32_TOL = 2e-5     # element-wise, relative to the field's max |value|
FP64_TOL = 1e-11


def rel_maxerr(got, ref):
    ref = np.asarray(ref)
    return float(np.max(np.abs(np.asarray(got) - ref)) / max(np.max(np.abs(ref)), 1e-300))


def half_spectrum(full):
    """(6, n1, n2, n3) full complex spectrum -> (6, n1, n2, n3//2+1)."""
    return full[..., : full.shape[-1] // 2 + 1]
