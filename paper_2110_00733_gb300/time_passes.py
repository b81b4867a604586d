"""Time the kernels of one MINRES iteration through hom_time_kernels.

    python -m paper_2110_00733_gb300.time_passes [--shape 256,256,256] [--reps 20]
                                                 [--staging 0|1] [--shape3 r,t2,t1] [--fp64]

Prints a JSON object {kernel: milliseconds} and each kernel's HBM rate from
its algorithmic bytes.  Used for launch-shape sweeps and, with --reps 1, as
a small driver for ncu captures of the pass kernels.
"""
from __future__ import annotations

import argparse
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2110_00733_gb300 import hom  # noqa: E402


def bytes_per_voxel(n3: int) -> dict:
    spec = 48.0 * (n3 // 2 + 1) / n3
    return {"x1_inv_gamma": 2 * spec, "x2_inv": 2 * spec, "x3_c2r_law_r2c": 2 * spec + 4,
            "x2_fwd": 2 * spec, "x1_fwd_gamma_dot": 3 * spec, "lanczos_update": 9 * spec}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--shape", default="256,256,256")
    ap.add_argument("--reps", type=int, default=20)
    ap.add_argument("--staging", type=int, default=0)
    ap.add_argument("--shape3", default="0,0,0")
    ap.add_argument("--fp64", action="store_true", help="FP64 fields (bytes below are for FP32)")
    a = ap.parse_args()
    shape = tuple(int(v) for v in a.shape.split(","))
    rng = np.random.default_rng(0)
    phi = (rng.random(shape) > 0.5).astype(np.float32)
    ctx = hom.hom_create(shape, phi, hom.HOM_INPUT_FRACTION_F32, 110e9, 0.3, staging=a.staging,
                         shape=tuple(int(v) for v in a.shape3.split(",")),
                         precision=hom.HOM_PREC_FP64 if a.fp64 else hom.HOM_PREC_FP32_FIELDS)
    t = hom.hom_time_kernels(ctx, reps=a.reps)
    ctx.close()
    V = int(np.prod(shape))
    bpv = {k: v * (2 if a.fp64 else 1) for k, v in bytes_per_voxel(shape[2]).items()}
    out = {"shape": shape, "ms": t,
           "gbs": {k: bpv[k] * V / (t[k] * 1e-3) / 1e9 for k in bpv if t.get(k, 0) > 0}}
    print(json.dumps(out))


if __name__ == "__main__":
    main()
