"""Learned warm start: training data from the solver itself, training on the
GPU with the library's network kernels, and warm-started versus zero-start
solves.

    python -m paper_2110_00733_gb300.warmstart [--train 2000] [--n 64]
        [--epochs 12] [--batch 8] [--eval 128,256] [--eval-cells 3]
        [--void-weight 1.0] [--save net.bin] [--load net.bin]

Training set (seed i): octet cell on an n^3 grid at density U[0.03, 0.30],
macro strain uniform on the Mandel unit sphere, FP32-field Galerkin-MINRES
to 1e-6; the target is the strain fluctuation.  Held-out cells (seeds 10000
and up) on finer grids: the network runs on the training grid (phi averaged
over s^3 blocks, s = N / n) and its head is interpolated back, then
hom_solve starts from the projected prediction.  Printed as JSON lines.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

E_M, NU_M = 110e9, 0.3


def make_dataset(n, count, seed0=0, rho_lo=0.03, rho_hi=0.30, tol=1e-6, max_it=6000):
    """Solver-generated pairs on the device: phi [count, V], macro [count, 6]
    (tensor components), target [count, 6, V] (strain fluctuation, tensor
    components)."""
    import torch
    import rve_inputs as ri
    from paper_2110_00733_gb300 import hom
    V = n ** 3
    fam = ri.OctetFamily(n)
    phi = torch.zeros((count, V), dtype=torch.float32, device="cuda")
    target = torch.zeros((count, 6, V), dtype=torch.float32, device="cuda")
    macro = np.zeros((count, 6))
    iters = []
    for i in range(count):
        rng = np.random.default_rng(seed0 + i)
        rho = rng.uniform(rho_lo, rho_hi)
        E = ri.unit_sphere_strain(rng)
        phi[i] = torch.from_numpy(fam.phi(rho).reshape(-1))
        with hom.hom_create((n, n, n), phi[i], hom.HOM_INPUT_FRACTION_F32, E_M, NU_M, device_ptrs=True) as ctx:
            rc, info = hom.hom_solve(ctx, E, tol=tol, max_it=max_it)
            hom.hom_fields(ctx, 0, strain=target[i], want=("strain",))
        target[i] -= torch.tensor(E, dtype=torch.float32, device="cuda")[:, None]
        macro[i] = E
        iters.append(info[0]["iterations"])
    torch.cuda.synchronize()
    return phi, macro, target, iters


def train(net, n, phi, macro, target, epochs=12, batch=8, lr_max=2e-3, lr_min=2e-5, seed=0, log=None):
    """Adam with a linear warm-up and cosine decay; returns the mean loss of
    each epoch."""
    import torch
    count = phi.shape[0]
    steps_per = count // batch
    total = epochs * steps_per
    warm = min(100, total // 10 + 1)
    rng = np.random.default_rng(seed)
    step = 0
    out = []
    for ep in range(epochs):
        perm = rng.permutation(count)
        acc = 0.0
        for b in range(steps_per):
            idx = perm[b * batch:(b + 1) * batch]
            it = torch.from_numpy(idx).cuda()
            lr = lr_max * min(1.0, (step + 1) / warm)
            if step >= warm:
                lr = lr_min + 0.5 * (lr_max - lr_min) * (1 + math.cos(math.pi * (step - warm) / max(1, total - warm)))
            acc += net.train_step((n, n, n), phi[it].contiguous(), macro[idx], target[it].contiguous(), lr)
            step += 1
        out.append(acc / steps_per)
        if log:
            log({"epoch": ep, "loss": out[-1], "lr": lr})
    return out


def evaluate(net, n_train, N, seeds, tol=1e-6, max_it=20000, fp64_baseline=False):
    """Zero-start and warm-started FP32 solves of held-out octet cells on an
    N^3 grid; times are wall clock of hom_solve (plus inference for the
    warm start)."""
    import torch
    import rve_inputs as ri
    from paper_2110_00733_gb300 import hom
    s = N // n_train
    rows = []
    for seed in seeds:
        rng = np.random.default_rng(seed)
        rho = rng.uniform(0.03, 0.30)
        E = ri.unit_sphere_strain(rng)
        phi_np, _ = ri.octet(N, rho)
        phi = torch.from_numpy(phi_np.reshape(-1)).cuda()
        row = {"N": N, "seed": seed, "rho": rho}
        with hom.hom_create((N, N, N), phi, hom.HOM_INPUT_FRACTION_F32, E_M, NU_M, device_ptrs=True) as ctx:
            hom.hom_solve(ctx, E, tol=tol, max_it=max_it)            # warm-up (graph capture)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            rc0, i0 = hom.hom_solve(ctx, E, tol=tol, max_it=max_it)
            torch.cuda.synchronize()
            t_zero = time.perf_counter() - t0
            x0 = torch.zeros((1, 6, N ** 3), dtype=torch.float32, device="cuda")
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            net.warm_start((N, N, N), s, phi, E, x0)
            t_inf = time.perf_counter() - t0
            rc1, i1 = hom.hom_solve(ctx, E, tol=tol, max_it=max_it, warm_start=x0)
            torch.cuda.synchronize()
            t_warm = time.perf_counter() - t0
        row.update(zero_it=i0[0]["iterations"], zero_s=t_zero, zero_res=i0[0]["true_residual"],
                   warm_it=i1[0]["iterations"], warm_s=t_warm, inference_s=t_inf, warm_res=i1[0]["true_residual"],
                   rc=(rc0, rc1),
                   sigma_rel_diff=float(np.max(np.abs(i1[0]["sigma_mean"] - i0[0]["sigma_mean"]))
                                        / np.max(np.abs(i0[0]["sigma_mean"]))))
        if fp64_baseline:
            with hom.hom_create((N, N, N), phi, hom.HOM_INPUT_FRACTION_F32, E_M, NU_M, device_ptrs=True,
                                precision=hom.HOM_PREC_FP64) as ctx:
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                rc2, i2 = hom.hom_solve(ctx, E, tol=tol, max_it=max_it)
                torch.cuda.synchronize()
                row.update(fp64_zero_it=i2[0]["iterations"], fp64_zero_s=time.perf_counter() - t0)
        rows.append(row)
    return rows


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--train", type=int, default=2000)
    ap.add_argument("--n", type=int, default=64)
    ap.add_argument("--epochs", type=int, default=12)
    ap.add_argument("--batch", type=int, default=8)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--eval", default="128,256")
    ap.add_argument("--eval-cells", type=int, default=3)
    ap.add_argument("--fp64-baseline", action="store_true")
    ap.add_argument("--void-weight", type=float, default=1.0,
                    help="loss weight of empty voxels (1: plain mean squared error)")
    ap.add_argument("--save", default=None)
    ap.add_argument("--load", default=None)
    a = ap.parse_args(argv)
    import torch
    from paper_2110_00733_gb300 import build, net as hnet
    build.build()
    torch.cuda.set_device(0)
    emit = lambda d: print(json.dumps(d), flush=True)   # noqa: E731
    model = hnet.Net(seed=1)
    model.set_void_weight(a.void_weight)
    emit({"params": model.param_count(), "void_weight": a.void_weight})
    if a.load:
        model.load(a.load)
    else:
        t0 = time.perf_counter()
        phi, macro, target, its = make_dataset(a.n, a.train)
        emit({"dataset": a.train, "n": a.n, "seconds": time.perf_counter() - t0, "mean_iterations": float(np.mean(its))})
        t0 = time.perf_counter()
        l0 = model.kernel_launches()
        losses = train(model, a.n, phi, macro, target, epochs=a.epochs, batch=a.batch, lr_max=a.lr, log=emit)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        emit({"train_seconds": dt, "epochs": a.epochs, "samples_per_s": a.epochs * (a.train // a.batch) * a.batch / dt,
              "final_loss": losses[-1], "kernel_launches": model.kernel_launches() - l0})
        # held-out loss at the training resolution
        hphi, hmacro, htarget, _ = make_dataset(a.n, 16, seed0=20000)
        x0 = torch.zeros_like(htarget)
        model.forward((a.n,) * 3, hphi, hmacro, x0)
        rel = float(torch.linalg.vector_norm(x0 - htarget) / torch.linalg.vector_norm(htarget))
        emit({"heldout_rel_error": rel})
        del phi, target
        if a.save:
            model.save(a.save)
    for N in [int(v) for v in a.eval.split(",") if v]:
        for row in evaluate(model, a.n, N, range(10000, 10000 + a.eval_cells), fp64_baseline=a.fp64_baseline):
            emit(row)
    model.close()


if __name__ == "__main__":
    main()
