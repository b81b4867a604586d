"""Time the kernels of one MINRES iteration through hom_time_kernels.

    python -m paper_2110_00733_gb300.time_passes [--shape 256,256,256] [--reps 20]

Prints a JSON object {kernel: milliseconds} and each kernel's HBM rate from
its algorithmic bytes (the per-kernel figures of the roofline table).  With
--reps 1 it is a small driver for ncu captures of the pass kernels:

    ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum,gpu__time_duration.sum \
        --clock-control none -k "regex:k_x" -c 24 --csv --log-file traffic.csv \
        python -m paper_2110_00733_gb300.time_passes --shape 256,128,256 --reps 1
    python -m paper_2110_00733_gb300.time_passes --traffic traffic.csv --shape 256,128,256

The second command turns the capture into profiles/traffic.json, which
bench.py reads while the solver's kernel sources are unchanged: the FP32
launches are kept (context creation runs three FP64 passes first), each
kernel of the iteration appears twice (warm-up and one timed launch) and the
first of each is used; the fused n1 pass appears four times (warm-up, then
three launches that cycle through the deferred x update) and the mean of the
last three is used.
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
    return {"x2_inv": 2 * spec, "x3_c2r_law_energy_r2c": 2 * spec + 4, "x2_fwd": 2 * spec,
            "x1_fwd_lanczos_inv": (8 + 2 / 3) * spec}   # x read and written on one step in three


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--shape", default="256,256,256")
    ap.add_argument("--reps", type=int, default=20)
    ap.add_argument("--traffic", default=None, help="ncu CSV to summarise into profiles/traffic.json")
    a = ap.parse_args()
    shape = tuple(int(v) for v in a.shape.split(","))
    if a.traffic:
        return write_traffic(a.traffic, shape)
    rng = np.random.default_rng(0)
    phi = (rng.random(shape) > 0.5).astype(np.float32)
    ctx = hom.hom_create(shape, phi, hom.HOM_INPUT_FRACTION_F32, 110e9, 0.3)
    t = hom.hom_time_kernels(ctx, reps=a.reps)
    ctx.close()
    V = int(np.prod(shape))
    bpv = bytes_per_voxel(shape[2])
    out = {"shape": shape, "ms": t,
           "gbs": {k: bpv[k] * V / (t[k] * 1e-3) / 1e9 for k in bpv if t.get(k, 0) > 0}}
    print(json.dumps(out))


# kernel launches of one MINRES iteration in hom_time_kernels order
ORDER = ["x2_inv", "x3_c2r_law_energy_r2c", "x2_fwd", "x1_fwd_lanczos_inv"]


def write_traffic(csv_path, shape):
    import csv
    rows = list(csv.reader(open(csv_path)))
    start = next(i for i, r in enumerate(rows) if "Kernel Name" in r)
    hdr = rows[start]
    ki, ii, mi, vi, ui = (hdr.index(k) for k in ("Kernel Name", "ID", "Metric Name", "Metric Value", "Metric Unit"))
    launches = {}
    for r in rows[start + 1:]:
        if len(r) <= vi:
            continue
        d = launches.setdefault(int(r[ii]), {"name": r[ki]})
        scale = {"byte": 1e-6, "Kbyte": 1e-3, "Mbyte": 1.0, "Gbyte": 1e3}.get(r[ui], 1.0)
        if r[mi].startswith("dram__bytes"):
            d[r[mi]] = float(r[vi].replace(",", "")) * scale
    seq = [launches[k] for k in sorted(launches) if "<double" not in launches[k]["name"]]
    # the first launch of each kernel of the step (hom_time_kernels launches
    # each twice: warm-up, then --reps 1; the fused n1 pass four times, see
    # below); FP64 launches of context creation and the first inverse n1 pass
    # are skipped
    patterns = {"x2_inv": ("k_x2_tma<float, 1,", "k_x2<float, 1,"), "x3_c2r_law_energy_r2c": ("k_x3r<", "k_x3<float"),
                "x2_fwd": ("k_x2_tma<float, -1,", "k_x2_tma<float, (int)-1", "k_x2<float, -1,", "k_x2<float, (int)-1"),
                "x1_fwd_lanczos_inv": ("k_x1_lanczos",)}
    firsts = []
    for name in ORDER:
        hits = [d for d in seq if any(d["name"].startswith(p) or (" " + p) in d["name"] for p in patterns[name])]
        d = hits[0] if hits else {"name": "(not captured)"}
        if name == "x1_fwd_lanczos_inv" and len(hits) >= 4:
            # one warm-up launch, then three that cycle through the steps of the
            # deferred x update (x read and written on one of them): their mean
            d = {"name": hits[1]["name"]}
            for m in ("dram__bytes_read.sum", "dram__bytes_write.sum"):
                d[m] = sum(h.get(m, 0.0) for h in hits[1:4]) / 3.0
        firsts.append(d)
    V = int(np.prod(shape))
    out = {"source_hash": source_hash(), "grid": list(shape),
           "capture": "ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum,gpu__time_duration.sum "
                      "--clock-control none -k \"regex:k_x\" -c 24 --csv --log-file traffic.csv "
                      f"python -m paper_2110_00733_gb300.time_passes --shape {','.join(map(str, shape))} --reps 1",
           "note": "bytes per voxel on this grid (work spectrum larger than L2); traffic scales with the voxel "
                   "count at fixed n3, so bench.py multiplies by n^3 for the 256^3 workload",
           "kernels": {}}
    for name, d in zip(ORDER, firsts):
        rd, wr = d.get("dram__bytes_read.sum", 0.0), d.get("dram__bytes_write.sum", 0.0)
        out["kernels"][name] = {"ncu_kernel": d["name"].split("(")[0], "dram_read_mb": round(rd, 1),
                                "dram_write_mb": round(wr, 1), "dram_bytes_per_voxel": (rd + wr) * 1e6 / V}
    path = os.path.join(ROOT, "profiles", "traffic.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out["kernels"], indent=1))
    return 0


def source_hash():
    """Hash of the solver's kernel sources (the network's files do not change
    the solver kernels' traffic)."""
    import hashlib
    h = hashlib.sha256()
    cdir = os.path.join(ROOT, "paper_2110_00733_gb300", "csrc")
    for fn in ("hom_fft.cuh", "hom_tma.cuh", "hom_passes.cuh", "hom_modb.cuh", "hom_internal.h",
               "hom_kernels_f32.cu", "hom_kernels_f64.cu"):
        with open(os.path.join(cdir, fn), "rb") as f:
            h.update(fn.encode())
            h.update(f.read())
    return h.hexdigest()[:16]


if __name__ == "__main__":
    sys.exit(main())
