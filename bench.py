"""Benchmark: Galerkin-FFT + MINRES homogenization of an octet-truss cell.

Workload (one step = one full solve through the C ABI): octet-truss unit cell
on a 256^3 periodic grid, relative density 10 %, Voigt volume fractions from
4^3 sub-voxel sampling, E = 110 GPa, nu = 0.3, rotated finite-difference
frequencies, macro strain E11 = 1e-3, FP32 fields with FP64 Krylov scalars,
tolerance 1e-6 on the FP64 true relative residual.  A step computes b, runs
MINRES to the tolerance, checks the FP64 true residual and forms the mean
stress.  Metric: MINRES voxel-iterations per second (V x iterations / time);
ms_per_step is the time to the 1e-6 residual.

Every field (403 MB per 6-component FP32 field) is larger than the 129 MB
L2, so no flush is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                    [--n 256] [--rho 0.10]

--impl reference times the FP64 CPU oracle (the reference arm of this
repository) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import itertools
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

E_M, NU_M = 110e9, 0.3
MACRO = np.array([1e-3, 0, 0, 0, 0, 0], dtype=np.float64)
TOL = 1e-6
MAX_IT = 20000

# Algorithmic bytes per voxel moved by each kernel of one MINRES iteration,
# FP32 fields: one half spectrum (6 complex64 per frequency) is
# 48 (n3/2+1)/n3 bytes per voxel; the MINRES vectors are half spectra too.
def kernel_bytes_per_voxel(n3: int) -> dict:
    spec = 48.0 * (n3 // 2 + 1) / n3
    return {
        "x2_inv": 2 * spec,                   # work spectrum in place
        "x3_c2r_law_energy_r2c": 2 * spec + 4,   # + phi
        "x2_fwd": 2 * spec,
        # read work, u_k, u_{k-1}, w_{k-2}, w_{k-3}; write u_{k+1}, w_{k-1},
        # work; x read and written on one step in three
        "x1_fwd_lanczos_inv": (8 + 2 / 3) * spec,
    }


# algorithmic minimum of one MINRES iteration (FP32 fields) with x read and
# written on every step; the fused step touches x on one step in three
ITER_BYTES_PER_VOXEL = 196.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--rho", type=float, default=0.10)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--host-loop", action="store_true",
                    help="replay the MINRES loop body from the host (same kernels; lets ncu list them)")
    ap.add_argument("--cpu-iters", type=int, default=2)
    ap.add_argument("--warm", action="store_true",
                    help="asprinted: also solve from the learned warm start (the network is trained first)")
    ap.add_argument("--train", type=int, default=2000, help="warm start: solver runs in the training set")
    ap.add_argument("--epochs", type=int, default=24, help="warm start: training epochs")
    ap.add_argument("--workload", default="headline",
                    choices=["headline", "modbfft", "batch", "config2", "asprinted", "uniaxial", "ablation",
                             "smoothing", "j2", "j2curve", "warmstart", "stacked"],
                    help="headline: the default line; modbfft: the same cell with the MoDBFFT solver; "
                         "batch: 16 octet cells x 6 unit strains at once; stacked: one against six "
                         "stacked load cases per grid size")
    return ap.parse_args()


def config(n, rho):
    return {"workload": f"octet_truss_{n}^3_rho{rho:.2f}_E11_tol1e-6",
            "grid": [n, n, n], "relative_density": rho, "voigt_subsamples": 64,
            "E_pa": E_M, "nu": NU_M, "derivative": "rotated", "macro_strain": "E11=1e-3",
            "fields": "fp32", "krylov_scalars": "fp64", "tol": TOL,
            "l2": "inputs larger than L2 (403 MB fields), no flush"}


# --------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (FileNotFoundError, OSError):
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.t:
            self.t.join(timeout=2)
        mhz, maxm, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                mhz.append(float(parts[1]))
                maxm.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not mhz:
            return None
        return {"sm_mhz": statistics.median(mhz), "sm_max_mhz": max(maxm),
                "reasons": sorted(reasons), "samples": len(mhz)}


# --------------------------------------------------------------------------- helpers
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def reduce_over_ranks(dist, t_local, units_local, device):
    """(max over ranks of the timed-region seconds, sum over ranks of the
    work units): the whole-job throughput is units / seconds.  Without a
    process group the local values."""
    if dist is None:
        return float(t_local), float(units_local)
    import torch
    t = torch.tensor([float(t_local)], dtype=torch.float64, device=device)
    u = torch.tensor([float(units_local)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def step_stats(step_ms, step_units):
    """Best and median over the timed solves: per-solve milliseconds (CUDA
    events on the library's stream between consecutive solves) and the
    voxel-iterations/s each solve gives.  None without a timed solve."""
    if not step_ms:
        return None
    rates = [u / (ms * 1e-3) for ms, u in zip(step_ms, step_units) if ms > 0]
    return {"n": len(step_ms), "best_ms": min(step_ms), "median_ms": statistics.median(step_ms),
            "best_voxel_iters_per_s": max(rates) if rates else None,
            "median_voxel_iters_per_s": statistics.median(rates) if rates else None}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def kernel_traffic(name, n):
    """DRAM bytes per launch of `name` from the committed ncu summary, scaled
    to an n^3 grid, or None when absent or taken on a different kernel source."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    k = d.get("kernels", {}).get(name)
    if not k:
        return None
    if d.get("source_hash") != source_hash():
        return None
    return k["dram_bytes_per_voxel"] * n ** 3


def oracle_error(n, rho, sigma_mean):
    """Error of this result's mean stress against the FP64 oracle's for the
    same cell and macro strain, solved to a relative residual of 1e-10 and
    stored in tests/golden/ by tests/golden/make_octet_golden.py (max abs
    difference over the 6 components / max |oracle|), or None when no stored
    value exists for this cell."""
    p = os.path.join(ROOT, "tests", "golden", f"octet{n}_rho{rho:.2f}.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        gold = json.load(f)
    for case in gold["cases"]:
        if np.allclose(case["macro_strain"], MACRO / np.max(np.abs(MACRO))):
            ref = np.asarray(case["sigma_mean"]) * np.max(np.abs(MACRO))   # linear in the macro strain
            err = float(np.max(np.abs(np.asarray(sigma_mean) - ref)) / np.max(np.abs(ref)))
            return {"rel_err_sigma_mean": err, "oracle_tol": gold["tol"],
                    "oracle_iterations": case["iterations"], "source": os.path.relpath(p, ROOT)}
    return None


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


# --------------------------------------------------------------------------- CPU oracle
def cpu_oracle_sample(phi64, iters):
    """Oracle Galerkin-MINRES on the same cell, capped at `iters` iterations
    (plus its right-hand side and true-residual operator applications)."""
    import oracle
    t0 = time.perf_counter()
    s = oracle.solve(phi64, E_M, NU_M, 1, MACRO, tol=1e-30, max_it=iters)
    dt = time.perf_counter() - t0
    return s["iterations"], dt, oracle.num_threads()


def j2_cpu_sample(phi64, E, nu, sy, H, e11, max_lin):
    """The oracle's J2 Newton step on the same cell: the first increment to
    e11 with lateral faces free, one Newton iteration whose MINRES solve is
    capped at max_lin iterations (its right-hand side, line search and
    history update included).  Returns (MINRES iterations, seconds, threads)."""
    import oracle
    cell = oracle.J2Cell(phi64, E, nu, sy, H)
    t0 = time.perf_counter()
    out = cell.increment(0b111110, [e11, 0, 0, 0, 0, 0], np.zeros(6), tol_lin=1e-30, max_newton=1,
                         max_lin=max_lin)
    dt = time.perf_counter() - t0
    return out["linear"], dt, oracle.num_threads()


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import rve_inputs as ri
    n = args.n
    phi, _ = ri.octet(n, args.rho)
    phi64 = phi.astype(np.float64)
    V = n ** 3
    for _ in range(args.warmup):
        cpu_oracle_sample(phi64, 1)
    tot_it, tot_t, cores = 0, 0.0, 1
    for _ in range(args.steps):
        it, dt, cores = cpu_oracle_sample(phi64, args.cpu_iters)
        tot_it += it
        tot_t += dt
    val = V * tot_it / tot_t
    sample = (f"{n}^3 octet rho={args.rho}: {args.cpu_iters} MINRES iterations per step plus the "
              f"right-hand side and true-residual operator applications, FP64 oracle")
    line = {"impl": "reference", "metric": "minres_voxel_iters_per_s", "value": val,
            "unit": "voxel-iter/s", "n_gpus": 0, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * tot_t / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": config(n, args.rho),
            "cpu_baseline": {"value": val, "unit": "voxel-iter/s", "cores": cores,
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": val, "unit": "voxel-iter/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------- GPU arm
def run_ours(args):
    import torch
    ws, rank, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist_mod
        dist_mod.init_process_group("nccl", device_id=torch.device("cuda", local))
        dist = dist_mod
    from paper_2110_00733_gb300 import build, hom
    build.build()
    import rve_inputs as ri

    n = args.n
    V = n ** 3
    phi, radius = ri.octet(n, args.rho)
    phi = np.ascontiguousarray(phi, dtype=np.float32)
    stream = torch.cuda.Stream()
    phi_dev = torch.from_numpy(phi).cuda()
    ctx = hom.hom_create(phi.shape, phi_dev, hom.HOM_INPUT_FRACTION_F32, E_M, NU_M,
                         derivative=hom.HOM_DERIV_ROTATED, precision=hom.HOM_PREC_FP32_FIELDS,
                         device_ptrs=True, stream=stream.cuda_stream, device=local, host_loop=args.host_loop)

    def barrier():
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    def step():
        rc, info = hom.hom_solve(ctx, MACRO, tol=TOL, max_it=MAX_IT)
        return rc, info[0]

    for _ in range(args.warmup):
        step()
    barrier()
    clocks = ClockSampler(local)
    clocks.start()
    l0 = hom.hom_kernel_launches(ctx)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    marks = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]   # after each solve
    barrier()
    ev0.record(stream)
    iters, infos, step_units = 0, [], []
    for i in range(args.steps):
        rc, inf = step()
        marks[i].record(stream)
        iters += inf["iterations"]
        step_units.append(V * inf["iterations"])
        infos.append(inf)
    ev1.record(stream)
    barrier()
    step_ms = [a.elapsed_time(b) for a, b in zip([ev0] + marks[:-1], marks)]
    launches = hom.hom_kernel_launches(ctx) - l0
    ms = ev0.elapsed_time(ev1)
    clk = clocks.stop()
    t_local = ms / 1e3
    t_max, units = reduce_over_ranks(dist, t_local, V * iters, "cuda")
    value = units / t_max

    # Roofline of the MINRES step as a whole: its algorithmic bytes (196 B
    # per voxel-iteration, the least an iteration can move with FP32 fields:
    # read v_k, phi, v_{k-1}, w_{k-1}, w_{k-2}, x, write v_{k+1}, w_k, x)
    # over the live time per iteration of the timed solves; the per-kernel
    # figures come from CUDA events on the library's stream
    # (hom_time_kernels) and explain it.
    ktimes = hom.hom_time_kernels(ctx, reps=20)
    kb = kernel_bytes_per_voxel(n)
    peak, peak_kind = measured_peaks()
    kernels = {}
    for k, b in kb.items():
        if ktimes.get(k, 0.0) > 0:
            gbs = b * V / (ktimes[k] * 1e-3) / 1e9
            kernels[k] = {"ms": ktimes[k], "bytes_per_voxel": b, "achieved_gbs": gbs, "frac": gbs / peak,
                          "traffic": kernel_traffic(k, n)}
    dom = max(kernels, key=lambda k: kernels[k]["ms"])
    iter_achieved = ITER_BYTES_PER_VOXEL * V * iters / t_local / 1e9
    step_traffic = [kernels[k]["traffic"] for k in kernels]
    roofline = {"bound": "hbm", "kernel": "minres_iteration", "achieved": iter_achieved, "peak": peak,
                "peak_source": peak_kind, "unit": "GB/s", "frac": iter_achieved / peak,
                "traffic": (sum(step_traffic) if all(t is not None for t in step_traffic) else None),
                "bytes_per_voxel": ITER_BYTES_PER_VOXEL,
                "moved_bytes_per_voxel": sum(kb.values()),
                "launch_sum_ms": sum(ktimes.values()),
                "iteration_ms": 1e3 * t_local / max(iters, 1),
                "dominant_kernel": dict(name=dom, **kernels[dom]),
                "kernels": kernels}

    # end-to-end through the C ABI with host buffers: create (phi H2D), solve,
    # read the mean stress back, destroy
    e2e_vals = []
    for _ in range(max(1, min(args.steps, 3))):
        barrier()
        t0 = time.perf_counter()
        c2 = hom.hom_create(phi.shape, phi, hom.HOM_INPUT_FRACTION_F32, E_M, NU_M,
                            derivative=hom.HOM_DERIV_ROTATED, device=local)
        rc, info = hom.hom_solve(c2, MACRO, tol=TOL, max_it=MAX_IT)
        _ = info[0]["sigma_mean"]
        c2.close()
        t1 = time.perf_counter()
        e2e_vals.append(V * info[0]["iterations"] / (t1 - t0))
    e2e = {"value": ws * statistics.median(e2e_vals), "unit": "voxel-iter/s",
           "h2d_bytes_per_step": int(phi.nbytes), "d2h_bytes_per_step": 6 * 8 + 64}

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        it, dt, cores = cpu_oracle_sample(phi.astype(np.float64), args.cpu_iters)
        cpu = {"value": V * it / dt, "unit": "voxel-iter/s", "cores": cores, "kind": "oracle",
               "sample": f"{n}^3 octet, {it} FP64 MINRES iterations plus rhs and true-residual "
                         f"applications ({dt:.1f} s)"}

    last = infos[-1]
    if rank == 0:
        line = {"metric": "minres_voxel_iters_per_s", "value": value, "unit": "voxel-iter/s",
                "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": 1e3 * t_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic octet-truss cell (seeded generator)",
                "config": dict(config(n, args.rho), parallelism=f"replicas{ws}",
                               **({"loop": "host-replayed body"} if args.host_loop else {})),
                "iterations_per_step": iters / args.steps,
                "time_to_tol_ms": 1e3 * t_max / args.steps,
                "step_ms": step_stats(step_ms, step_units),
                "true_residual": last["true_residual"], "sweeps": last["sweeps"],
                "sigma11_pa": float(last["sigma_mean"][0]),
                "vs_fp64_oracle": oracle_error(n, args.rho, last["sigma_mean"]),
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": int(launches), "clocks": clk}
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist:
        dist.destroy_process_group()
    return 0


def run_batch(args):
    """16 octet cells, densities uniform in [0.03, 0.30], grids drawn from
    {64, 96, 128, 160}^3 (seeds 0-15), six unit strains each, solved at once
    by hom_solve_batch with autotuned launch shapes; FP32 fields, tol 1e-6.
    Value: sum over cells and cases of V x iterations / wall time."""
    import torch
    from paper_2110_00733_gb300 import build, hom
    build.build()
    import rve_inputs as ri
    torch.cuda.set_device(0)
    rng = np.random.default_rng(0)
    specs = [(int(rng.choice([64, 96, 128, 160])), float(rng.uniform(0.03, 0.30))) for _ in range(16)]
    phis = [ri.octet(n, rho)[0] for n, rho in specs]
    ctxs = [hom.hom_create(p.shape, p, hom.HOM_INPUT_FRACTION_F32, E_M, NU_M, autotune=True) for p in phis]
    macros = np.eye(6)
    for _ in range(args.warmup):
        hom.hom_solve_batch(ctxs, macros, tol=TOL, max_it=MAX_IT)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    vox_it = 0
    for _ in range(args.steps):
        rc, infos = hom.hom_solve_batch(ctxs, macros, tol=TOL, max_it=MAX_IT)
        for (n, _), cell in zip(specs, infos):
            vox_it += n ** 3 * sum(i["iterations"] for i in cell)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    worst = max(i["true_residual"] for cell in infos for i in cell)
    print(json.dumps({"metric": "minres_voxel_iters_per_s", "value": vox_it / dt, "unit": "voxel-iter/s",
                      "workload": "batch_16_octet_cells_x6", "cells": specs, "steps": args.steps,
                      "ms_per_step": 1e3 * dt / args.steps, "worst_true_residual": worst,
                      "iterations": [[i["iterations"] for i in cell] for cell in infos]}), flush=True)
    for c in ctxs:
        c.close()
    return 0


def run_stacked(args):
    """One load case (E11) against the six unit strains stacked in one
    hom_solve, octet cells at rho = 0.15 on grids 64, 96, 128, 160, 256;
    FP32 fields, tol 1e-6, one warm-up solve, then one timed (wall clock).
    One line per grid and case count."""
    import torch
    from paper_2110_00733_gb300 import build, hom
    build.build()
    import rve_inputs as ri
    torch.cuda.set_device(0)
    for n in (64, 96, 128, 160, 256):
        phi, _ = ri.octet(n, 0.15)
        for ncase in (1, 6):
            ctx = hom.hom_create(phi.shape, phi, hom.HOM_INPUT_FRACTION_F32, E_M, NU_M)
            macros = np.eye(6)[:ncase]
            hom.hom_solve(ctx, macros, tol=TOL, max_it=MAX_IT)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            rc, info = hom.hom_solve(ctx, macros, tol=TOL, max_it=MAX_IT)
            dt = time.perf_counter() - t0
            it = sum(i["iterations"] for i in info)
            print(json.dumps({"metric": "minres_voxel_iters_per_s", "value": n ** 3 * it / dt,
                              "unit": "voxel-iter/s", "workload": f"stacked_octet_{n}^3_rho0.15_x{ncase}",
                              "rc": rc, "iterations": it, "s": dt,
                              "worst_true_residual": max(i["true_residual"] for i in info)}), flush=True)
            ctx.close()
    return 0


def run_modbfft(args):
    """The headline cell solved with MoDBFFT (section 2.2): PCG iterations."""
    import torch
    from paper_2110_00733_gb300 import build, hom
    build.build()
    import rve_inputs as ri
    torch.cuda.set_device(0)
    n = args.n
    phi, _ = ri.octet(n, args.rho)
    ctx = hom.hom_create(phi.shape, phi, hom.HOM_INPUT_FRACTION_F32, E_M, NU_M,
                         derivative=hom.HOM_DERIV_CONTINUOUS, solver=hom.HOM_SOLVER_MODBFFT_CG)
    for _ in range(args.warmup):
        hom.hom_solve(ctx, MACRO, tol=TOL, max_it=MAX_IT)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    its = 0
    for _ in range(args.steps):
        rc, info = hom.hom_solve(ctx, MACRO, tol=TOL, max_it=MAX_IT)
        its += info[0]["iterations"]
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    print(json.dumps({"metric": "pcg_voxel_iters_per_s", "value": n ** 3 * its / dt, "unit": "voxel-iter/s",
                      "workload": f"modbfft_octet_{n}^3_rho{args.rho:.2f}_E11_tol1e-6", "rc": rc,
                      "iterations_per_step": its / args.steps, "ms_per_step": 1e3 * dt / args.steps,
                      "true_residual": info[0]["true_residual"], "sweeps": info[0]["sweeps"],
                      "sigma11_pa": float(info[0]["sigma_mean"][0])}), flush=True)
    ctx.close()
    return 0


def run_uniaxial(args):
    """Mixed macroscopic control on the headline cell (eq. galop): uniaxial
    stress (all six components stress-controlled, s11 = 1 MPa) gives E and nu
    from one solve; they are compared with E = 1/S11 and nu = -S21/S11 of the
    compliance from six strain-controlled solves, and with a prescribed e11
    whose lateral faces are stress-free.  FP32 fields, tol 1e-6; the
    uniaxial-stress solve also runs once with FP64 fields."""
    import numpy as np
    import torch
    from paper_2110_00733_gb300 import build, hom
    build.build()
    import rve_inputs as ri
    torch.cuda.set_device(0)
    n = args.n
    phi, _ = ri.octet(n, args.rho)
    s11 = 1.0e6
    Sbar = np.array([[s11, 0, 0, 0, 0, 0]])
    zero = np.zeros((1, 6))
    out = {"metric": "mixed_control_voxel_iters_per_s", "unit": "voxel-iter/s",
           "workload": f"uniaxial_stress_octet_{n}^3_rho{args.rho:.2f}_tol1e-6"}
    with hom.hom_create(phi.shape, phi, hom.HOM_INPUT_FRACTION_F32, E_M, NU_M) as ctx:
        rc, info = hom.hom_solve(ctx, np.eye(6), tol=TOL, max_it=MAX_IT)
        S = np.linalg.inv(hom.hom_effective_stiffness(ctx))
        out["strain_control"] = {"E_pa": 1.0 / S[0, 0], "nu": -S[1, 0] / S[0, 0],
                                 "iterations": [i["iterations"] for i in info]}
        for _ in range(args.warmup):
            hom.hom_solve_mixed(ctx, zero, Sbar, 63, tol=TOL, max_it=MAX_IT)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        its = 0
        for _ in range(args.steps):
            rc, info = hom.hom_solve_mixed(ctx, zero, Sbar, 63, tol=TOL, max_it=MAX_IT)
            its += info[0]["iterations"]
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        e = info[0]["eps_mean"]
        out.update({"value": n ** 3 * its / dt, "ms_per_step": 1e3 * dt / args.steps, "rc": rc,
                    "iterations_per_step": its / args.steps, "sweeps": info[0]["sweeps"],
                    "true_residual": info[0]["true_residual"],
                    "uniaxial_stress": {"E_pa": s11 / e[0], "nu": -e[1] / e[0],
                                        "sigma_mean_pa": [float(v) for v in info[0]["sigma_mean"]]}})
        rc2, info2 = hom.hom_solve_mixed(ctx, np.array([[1e-3, 0, 0, 0, 0, 0]]), zero, 62, tol=TOL, max_it=MAX_IT)
        e2 = info2[0]["eps_mean"]
        out["free_lateral_faces"] = {"E_pa": info2[0]["sigma_mean"][0] / e2[0], "nu": -e2[1] / e2[0],
                                     "iterations": info2[0]["iterations"], "rc": rc2}
    with hom.hom_create(phi.shape, phi, hom.HOM_INPUT_FRACTION_F32, E_M, NU_M,
                        precision=hom.HOM_PREC_FP64) as ctx:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rc3, info3 = hom.hom_solve_mixed(ctx, zero, Sbar, 63, tol=TOL, max_it=MAX_IT)
        torch.cuda.synchronize()
        e3 = info3[0]["eps_mean"]
        out["uniaxial_stress_fp64"] = {"E_pa": s11 / e3[0], "nu": -e3[1] / e3[0],
                                       "iterations": info3[0]["iterations"], "rc": rc3,
                                       "ms": 1e3 * (time.perf_counter() - t0)}
    print(json.dumps(out), flush=True)
    return 0


def run_j2(args):
    """Elastoplastic octet (section 2.1.1 Newton extension, J2 material of
    section 5 with hardening E/100): uniaxial compression in e11, lateral
    mean stresses zero, four increments of -2.5e-3 with the default Newton
    tolerances (tol_lin 1e-6, tol_newton 5e-3), once with FP32 fields (Newton
    systems by FP32 MINRES, strains, history and residuals FP64) and once
    with FP64 fields.  The cell is 64^3 unless --n asks for a smaller one.
    value: MINRES iterations of the tangent systems times voxels per second
    of the increments' device time, from the faster run whose increments
    all converged."""
    import numpy as np
    import torch
    from paper_2110_00733_gb300 import build, hom
    build.build()
    import rve_inputs as ri
    torch.cuda.set_device(0)
    n = min(args.n, 64)
    phi, _ = ri.octet(n, args.rho)
    sy, H = 70e6, E_M / 100
    out = {"metric": "j2_newton_voxel_iters_per_s", "unit": "voxel-iter/s",
           "workload": f"j2_octet_{n}^3_rho{args.rho:.2f}_uniaxial_e11_4x-2.5e-3_H=E/100"}
    for name, prec in (("fp32_fields", hom.HOM_PREC_FP32_FIELDS), ("fp64", hom.HOM_PREC_FP64)):
        run = {"increments": []}
        with hom.hom_create(phi.shape, phi, hom.HOM_INPUT_FRACTION_F32, E_M, NU_M, precision=prec,
                            host_loop=args.host_loop) as ctx:
            hom.hom_j2_begin(ctx, sy, H)
            hom.hom_j2_increment(ctx, [-1e-4, 0, 0, 0, 0, 0], np.zeros(6), 0b111110)   # warm-up (elastic)
            hom.hom_j2_begin(ctx, sy, H)
            launches0 = hom.hom_kernel_launches(ctx)
            lin, ms = 0, 0.0
            for k in range(1, 5):
                rc, info = hom.hom_j2_increment(ctx, [-2.5e-3 * k, 0, 0, 0, 0, 0], np.zeros(6), 0b111110,
                                                max_newton=60)
                lin += info["linear"]
                ms += info["time_ms"]
                run["increments"].append({"e11": -2.5e-3 * k, "rc": rc, "newton": info["newton"],
                                          "linear": info["linear"], "backtracks": info["backtracks"],
                                          "r_newton": info["r_newton"], "ms": info["time_ms"],
                                          "sigma11_pa": info["sigma_mean"][0],
                                          "lateral_over_axial": float(np.max(np.abs(info["sigma_mean"][1:])) /
                                                                      abs(info["sigma_mean"][0]))})
            _, _, alpha = hom.hom_j2_state(ctx)
            # kernel times at the last iterate (CUDA events on the library's stream)
            run["kernel_ms"] = hom.hom_j2_time_kernels(ctx, reps=20)
            run.update({"voxel_iters_per_s": n ** 3 * lin / (ms / 1e3), "ms_total": ms, "linear_total": lin,
                        "gpu_launches": hom.hom_kernel_launches(ctx) - launches0,
                        "yielded_fraction_of_struts": float((alpha[phi > 0.5] > 0).mean())})
        out[name] = run
    lin_cpu, dt_cpu, cores = j2_cpu_sample(phi.astype(np.float64), E_M, NU_M, sy, H, -2.5e-3, 20)
    out["cpu_baseline"] = {"value": n ** 3 * lin_cpu / dt_cpu, "unit": "voxel-iter/s", "cores": cores,
                           "kind": "oracle",
                           "sample": f"{n}^3, first increment, one Newton iteration with {lin_cpu} FP64 "
                                     f"MINRES iterations plus residuals and line search ({dt_cpu:.1f} s)"}
    # the line's value: the faster of the runs whose increments all converged
    ok = [k for k in ("fp32_fields", "fp64") if all(i["rc"] == 0 for i in out[k]["increments"])]
    best = min(ok, key=lambda k: out[k]["ms_total"]) if ok else "fp64"
    out["value"] = out[best]["voxel_iters_per_s"]
    out["value_from"] = best
    # roofline of the tangent application (the J2 kernel inside every MINRES
    # iteration): algorithmic bytes = the 36-entry tangent, the input and the
    # output strain per voxel, in the operator's precision.  At 64^3 the
    # tangent (38 MB in FP32) stays in L2 between back-to-back launches, so
    # the kernels are timed on a 128^3 cell (302 MB of tangent, larger than
    # L2), on its virgin state (an elastic return at every voxel)
    peak, peak_kind = measured_peaks()
    nt = 128
    phit, _ = ri.octet(nt, args.rho)
    prec_t = hom.HOM_PREC_FP32_FIELDS if best == "fp32_fields" else hom.HOM_PREC_FP64
    with hom.hom_create(phit.shape, phit, hom.HOM_INPUT_FRACTION_F32, E_M, NU_M, precision=prec_t) as ctx:
        hom.hom_j2_begin(ctx, sy, H)
        kms = hom.hom_j2_time_kernels(ctx, reps=20)
    w = 4 if best == "fp32_fields" else 8
    b_apply = (36 + 12) * w                          # tangent, input and output strain
    b_return = 8 * (6 + 6 + 1 + 6) + 36 * w + 8     # eps, epsp, alpha, sig (FP64), tangent, phi
    ach = b_apply * nt ** 3 / (kms["j2_tangent_apply"] * 1e-3) / 1e9
    out["roofline"] = {"bound": "hbm", "kernel": "j2_tangent_apply", "grid": [nt] * 3, "achieved": ach, "peak": peak,
                       "peak_source": peak_kind, "unit": "GB/s", "frac": ach / peak, "traffic": None,
                       "bytes_per_voxel": b_apply, "kernel_ms": kms,
                       "j2_return": {"bytes_per_voxel": b_return, "ms": kms["j2_return"],
                                     "achieved_gbs": b_return * nt ** 3 / (kms["j2_return"] * 1e-3) / 1e9}}
    out["dtype"] = "f32" if best == "fp32_fields" else "f64"
    print(json.dumps(out), flush=True)
    return 0


def run_j2curve(args):
    """Compression curves of section 5: octets of relative density 10, 20
    and 30 % at about 15 voxels per strut diameter (grids 160, 108 and 90;
    --n caps them), the lattice material of sections 4 and 5 (PA12: E =
    1.7 GPa, nu = 0.4; J2 perfect plasticity, yield stress 70 MPa), uniaxial
    compression to e11 = -10 % in 20 increments with free lateral faces,
    Newton tolerance 5e-3, FP32 fields.  One JSON line per increment,
    printed as it completes."""
    import numpy as np
    import torch
    from paper_2110_00733_gb300 import build, hom
    build.build()
    import rve_inputs as ri
    torch.cuda.set_device(0)
    e_pa12, nu_pa12, sy = 1.7e9, 0.4, 70e6
    for rho, n_full in ((0.10, 160), (0.20, 108), (0.30, 90)):
        n = min(args.n, n_full)
        phi, _ = ri.octet(n, rho)
        with hom.hom_create(phi.shape, phi, hom.HOM_INPUT_FRACTION_F32, e_pa12, nu_pa12,
                            host_loop=args.host_loop) as ctx:
            hom.hom_j2_begin(ctx, sy, 0.0)
            for k in range(1, 21):
                e = -0.005 * k
                rc, info = hom.hom_j2_increment(ctx, [e, 0, 0, 0, 0, 0], np.zeros(6), 0b111110, max_newton=40)
                print(json.dumps({"workload": f"j2_curve_octet_{n}^3_rho{rho:.2f}_pa12_perfect_plasticity_fp32_fields",
                                  "e11": e, "rc": rc, "sigma11_pa": float(info["sigma_mean"][0]),
                                  "newton": info["newton"], "linear": info["linear"],
                                  "ms": info["time_ms"]}), flush=True)
    return 0


def run_ablation(args):
    """Krylov solver and frequency scheme (section 2.1): MINRES and CG on the
    Galerkin system, rotated and continuous frequencies, on octet cells with
    void and with the void filled by a 5 % phase; iterations and time to
    1e-6, max_it 5000, FP32 fields, and FP64 fields as well on the cells with
    void."""
    import numpy as np
    import torch
    from paper_2110_00733_gb300 import build, hom
    build.build()
    import rve_inputs as ri
    torch.cuda.set_device(0)
    n = args.n if args.n != 256 else 128
    for rho in (0.10, 0.20):
        phi, _ = ri.octet(n, rho)
        for fill in (0.0, 0.05):
            ph = (fill + (1.0 - fill) * phi).astype(np.float32)
            rows = {}
            precs = [("fp32", hom.HOM_PREC_FP32_FIELDS)] + ([("fp64", hom.HOM_PREC_FP64)] if fill == 0.0 else [])
            for (pname, prec), (deriv, dname), (solver, sname) in itertools.product(
                    precs, ((hom.HOM_DERIV_ROTATED, "rotated"), (hom.HOM_DERIV_CONTINUOUS, "continuous")),
                    ((hom.HOM_SOLVER_GALERKIN_MINRES, "minres"), (hom.HOM_SOLVER_GALERKIN_CG, "cg"))):
                with hom.hom_create(ph.shape, ph, hom.HOM_INPUT_FRACTION_F32, E_M, NU_M, derivative=deriv,
                                    solver=solver, precision=prec) as ctx:
                    hom.hom_solve(ctx, MACRO, tol=TOL, max_it=200)          # graph capture, warm-up
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    rc, info = hom.hom_solve(ctx, MACRO, tol=TOL, max_it=5000)
                    torch.cuda.synchronize()
                    rows[f"{sname}_{dname}_{pname}"] = {
                        "rc": rc, "iterations": info[0]["iterations"], "sweeps": info[0]["sweeps"],
                        "true_residual": info[0]["true_residual"], "ms": 1e3 * (time.perf_counter() - t0),
                        "sigma11_pa": float(info[0]["sigma_mean"][0])}
            print(json.dumps({"workload": f"ablation_octet_{n}^3_rho{rho:.2f}_fill{fill:.2f}_E11_tol1e-6", **rows}),
                  flush=True)
    return 0


def run_smoothing(args):
    """Phase maps of section 3 on one octet (rho = 0.15, 128^3 simulation
    grid): plain voxels (PV: the indicator at voxel centres), the Voigt rule
    on a 4^3 sub-grid (VFG), Voigt analytic (VA), phase-field smoothening of
    the indicator on the 2x finer grid with l = half a coarse voxel (PFS),
    and PFS of the VA map (CS).  Each map gets one uniaxial-stress solve
    (hom_solve_mixed, FP32 fields, tol 1e-6): E, nu, iterations, time."""
    import numpy as np
    import torch
    from paper_2110_00733_gb300 import build, hom
    build.build()
    import rve_inputs as ri
    torch.cuda.set_device(0)
    n, rho = 128, 0.15
    vfg, r = ri.octet(n, rho)
    d = ri.octet_center_distance(n).astype(np.float64)
    maps = {"PV": (d < r).astype(np.float64), "VFG": vfg.astype(np.float64), "VA": ri.va_phase(r - d, 1.0 / n)}
    df = ri.octet_center_distance(2 * n).astype(np.float64)
    omega = (df < r).astype(np.uint8)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    maps["PFS"] = hom.hom_pfs(omega, 2, 1.0, 1.0, 0.05)
    torch.cuda.synchronize()
    pfs_ms = 1e3 * (time.perf_counter() - t0)
    maps["CS"] = hom.hom_pfs(maps["VA"], 1, 0.5, 1.0, 0.05)
    out = {"workload": f"smoothing_octet_{n}^3_rho{rho:.2f}_uniaxial_stress_tol1e-6", "pfs_fine_grid": [2 * n] * 3,
           "pfs_ms": pfs_ms}
    Sbar = np.array([[1.0e6, 0, 0, 0, 0, 0]])
    for name, phi in maps.items():
        with hom.hom_create(phi.shape, np.ascontiguousarray(phi, dtype=np.float64), hom.HOM_INPUT_FRACTION_F64,
                            E_M, NU_M) as ctx:
            hom.hom_solve_mixed(ctx, np.zeros((1, 6)), Sbar, 63, tol=TOL, max_it=200)     # warm-up
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            rc, info = hom.hom_solve_mixed(ctx, np.zeros((1, 6)), Sbar, 63, tol=TOL, max_it=MAX_IT)
            torch.cuda.synchronize()
            e = info[0]["eps_mean"]
            out[name] = {"mean_phi": float(phi.mean()), "E_pa": 1.0e6 / e[0], "nu": -e[1] / e[0], "rc": rc,
                         "iterations": info[0]["iterations"], "ms": 1e3 * (time.perf_counter() - t0)}
    print(json.dumps(out), flush=True)
    return 0


def run_config2(args):
    """Octet cells at 128^3, densities {3, 7, 15, 30} %, both solvers
    (Galerkin-MINRES with rotated frequencies; MoDBFFT-PCG with continuous
    frequencies, alpha = 1e-4 E), FP64 fields versus FP32 fields with FP64
    Krylov scalars, six unit strains -> the 6x6 effective stiffness.  One JSON
    line per (density, solver) with both precisions and their difference."""
    import torch
    from paper_2110_00733_gb300 import build, hom
    build.build()
    import rve_inputs as ri
    torch.cuda.set_device(0)
    n = 128
    for rho in (0.03, 0.07, 0.15, 0.30):
        phi, _ = ri.octet(n, rho)
        for solver, deriv, name in ((hom.HOM_SOLVER_GALERKIN_MINRES, hom.HOM_DERIV_ROTATED, "galerkin_minres"),
                                    (hom.HOM_SOLVER_MODBFFT_CG, hom.HOM_DERIV_CONTINUOUS, "modbfft_pcg")):
            res = {}
            for prec, pname in ((hom.HOM_PREC_FP64, "fp64"), (hom.HOM_PREC_FP32_FIELDS, "fp32")):
                ctx = hom.hom_create(phi.shape, phi, hom.HOM_INPUT_FRACTION_F32, E_M, NU_M, derivative=deriv,
                                     precision=prec, solver=solver)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                rc, info = hom.hom_solve(ctx, np.eye(6), tol=TOL, max_it=6000)
                torch.cuda.synchronize()
                dt = time.perf_counter() - t0
                C = hom.hom_effective_stiffness(ctx)
                ctx.close()
                res[pname] = {"rc": rc, "seconds": dt, "iterations": [i["iterations"] for i in info],
                              "true_residual_max": max(i["true_residual"] for i in info),
                              "C11_pa": C[0, 0], "C12_pa": C[0, 1], "C44_pa": C[3, 3], "C": C}
            err = float(np.max(np.abs(res["fp32"]["C"] - res["fp64"]["C"])) / np.max(np.abs(res["fp64"]["C"])))
            for v in res.values():
                v.pop("C")
            print(json.dumps({"workload": f"config2_octet_128^3_rho{rho:.2f}", "solver": name,
                              "fp32_vs_fp64_Ceff_rel_err": err, **res}), flush=True)
    return 0


def run_asprinted(args):
    """Synthetic as-printed lattice: 2x2x2 octet cells at 512^3 (134 M voxels),
    12 % density, strut surface moved by a Gaussian random field (correlation
    3 voxels, std 1 voxel), spherical pores (radius 2-8 voxels, 1 % of the
    solid), Voigt fractions; FP32 fields, six unit strains stacked, tol 1e-6.
    With --warm the warm-start network is trained on solver runs at 64^3
    (one unit cell, as in warmstart.py), runs on a 128^3 grid (64 voxels per
    unit cell, phi averaged over 4^3 blocks) and its prediction starts the
    same six solves; both lines are printed."""
    import torch
    from paper_2110_00733_gb300 import build, hom
    build.build()
    import rve_inputs as ri
    torch.cuda.set_device(0)
    t0 = time.perf_counter()
    phi, r = ri.as_printed(args.n, cells=2, rho=0.12, seed=0)
    tgen = time.perf_counter() - t0
    V = args.n ** 3
    phi_d = torch.from_numpy(np.ascontiguousarray(phi, dtype=np.float32)).cuda()
    wl = f"as_printed_2x2x2_octet_{args.n}^3_rho0.12"
    with hom.hom_create(phi.shape, phi_d, hom.HOM_INPUT_FRACTION_F32, E_M, NU_M, device_ptrs=True) as ctx:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rc, info = hom.hom_solve(ctx, np.eye(6), tol=TOL, max_it=MAX_IT)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        C0 = hom.hom_effective_stiffness(ctx)
        its = [i["iterations"] for i in info]
        print(json.dumps({"workload": wl, "start": "zero", "rc": rc, "generation_s": tgen,
                          "phi_mean": float(phi.mean()), "solve_s": dt, "iterations": its,
                          "voxel_iters_per_s": V * sum(its) / dt,
                          "true_residual_max": max(i["true_residual"] for i in info),
                          "C_eff_pa": C0.tolist()}), flush=True)
        if not args.warm:
            return 0
        from paper_2110_00733_gb300 import net as hnet
        from paper_2110_00733_gb300 import warmstart as ws
        model = hnet.Net(seed=1)
        t0 = time.perf_counter()
        tphi, tmacro, ttarget, _ = ws.make_dataset(64, args.train)
        tdata = time.perf_counter() - t0
        t0 = time.perf_counter()
        losses = ws.train(model, 64, tphi, tmacro, ttarget, epochs=args.epochs)
        torch.cuda.synchronize()
        ttrain = time.perf_counter() - t0
        del tphi, ttarget
        x0 = torch.zeros((6, 6, V), dtype=torch.float32, device="cuda")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        model.warm_start((args.n,) * 3, args.n // 128, phi_d.reshape(-1), np.eye(6), x0)
        torch.cuda.synchronize()
        tinf = time.perf_counter() - t0
        rc, infow = hom.hom_solve(ctx, np.eye(6), tol=TOL, max_it=MAX_IT, warm_start=x0)
        torch.cuda.synchronize()
        dtw = time.perf_counter() - t0
        Cw = hom.hom_effective_stiffness(ctx)
        itw = [i["iterations"] for i in infow]
        print(json.dumps({"workload": wl, "start": "learned warm start", "rc": rc,
                          "dataset_s": tdata, "train_s": ttrain, "final_loss": losses[-1],
                          "inference_s": tinf, "solve_s_with_inference": dtw, "iterations": itw,
                          "voxel_iters_per_s": V * sum(itw) / dtw,
                          "true_residual_max": max(i["true_residual"] for i in infow),
                          "C_eff_rel_diff_vs_zero_start": float(np.max(np.abs(Cw - C0)) / np.max(np.abs(C0))),
                          "C_eff_pa": Cw.tolist()}), flush=True)
        model.close()
    return 0


def run_warmstart(args):
    """Learned warm start against zero start (config 4): the network is
    trained on --train solver runs at 64^3 (octet, density U[0.03, 0.30],
    macro strain uniform on the Mandel unit sphere), then on held-out octet
    cells at --n^3 (seeds 10000+, 8 unless --steps asks for more) each cell
    is solved from a zero start and from the network's prediction (network on
    64^3, phi averaged over (n/64)^3 blocks, head interpolated back), FP32
    fields, tol 1e-6 on the FP64 true residual.  Time to tolerance of the
    warm start includes inference.  One JSON line with the per-cell rows and
    the median savings."""
    import torch
    from paper_2110_00733_gb300 import build, net as hnet, warmstart as ws
    build.build()
    torch.cuda.set_device(0)
    model = hnet.Net(seed=1)
    t0 = time.perf_counter()
    tphi, tmacro, ttarget, its = ws.make_dataset(64, args.train)
    tdata = time.perf_counter() - t0
    t0 = time.perf_counter()
    losses = ws.train(model, 64, tphi, tmacro, ttarget, epochs=args.epochs)
    torch.cuda.synchronize()
    ttrain = time.perf_counter() - t0
    del tphi, ttarget
    ncell = max(8, args.steps)
    rows = ws.evaluate(model, 64, args.n, range(10000, 10000 + ncell))
    model.close()
    it_save = [1.0 - r["warm_it"] / r["zero_it"] for r in rows]
    t_save = [1.0 - r["warm_s"] / r["zero_s"] for r in rows]
    print(json.dumps({"metric": "time_to_tol_saving_learned_warm_start", "unit": "fraction",
                      "workload": f"warm_start_octet_{args.n}^3_heldout_x{ncell}_trained_64^3_x{args.train}",
                      "value": statistics.median(t_save), "median_iteration_saving": statistics.median(it_save),
                      "dataset_s": tdata, "train_s": ttrain, "final_loss": losses[-1],
                      "mean_train_iterations": float(np.mean(its)), "cells": rows}), flush=True)
    return 0


def main():
    args = parse()
    if args.workload == "config2":
        return run_config2(args)
    if args.workload == "asprinted":
        return run_asprinted(args)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch":
        return run_batch(args)
    if args.workload == "uniaxial":
        return run_uniaxial(args)
    if args.workload == "ablation":
        return run_ablation(args)
    if args.workload == "smoothing":
        return run_smoothing(args)
    if args.workload == "j2":
        return run_j2(args)
    if args.workload == "j2curve":
        return run_j2curve(args)
    if args.workload == "modbfft":
        return run_modbfft(args)
    if args.workload == "warmstart":
        return run_warmstart(args)
    if args.workload == "stacked":
        return run_stacked(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
