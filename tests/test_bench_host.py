"""Host logic of bench.py, on CPU: two gloo ranks (spawned processes,
127.0.0.1) that time different regions and process different amounts of
work reduce to the slowest rank's time and the summed work; the reference
arm prints on rank 0 only; the bounded oracle sample beside the j2 line
counts what it ran."""
import io
import contextlib
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ws, r, local = bench.dist_env()
        t, u = bench.reduce_over_ranks(dist, [1.5, 2.25][rank], [1000.0, 3000.0][rank], "cpu")
        dist.barrier()
        q.put((rank, ws, r, local, t, u))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_to_max_time_and_summed_work():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs)
    got = sorted(q.get(timeout=5) for _ in range(2))
    for rank, (r0, ws, r, local, t, u) in enumerate(got):
        assert (r0, ws, r, local) == (rank, 2, rank, rank)
        assert t == 2.25 and u == 4000.0


def test_single_process_reduction_is_the_identity():
    import bench
    assert bench.reduce_over_ranks(None, 0.5, 123.0, "cpu") == (0.5, 123.0)


@pytest.mark.parametrize("rank", [0, 1])
def test_reference_arm_prints_one_line_on_rank_zero_only(monkeypatch, rank):
    import json
    import bench
    monkeypatch.setenv("RANK", str(rank))
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--gpus", "2", "--n", "8",
                                      "--steps", "1", "--warmup", "0"])
    args = bench.parse()
    out = io.StringIO()
    with contextlib.redirect_stdout(out):
        assert bench.run_reference(args) == 0
    lines = out.getvalue().splitlines()
    if rank:
        assert lines == []
    else:
        assert len(lines) == 1
        line = json.loads(lines[0])
        assert line["impl"] == "reference" and line["value"] > 0
        assert line["cpu_baseline"]["kind"] == "oracle" and line["e2e"]["value"] == line["value"]


def test_j2_cpu_sample_counts_the_oracle_minres_iterations():
    """the bounded oracle sample beside the j2 bench line runs one Newton
    iteration with at most max_lin MINRES iterations"""
    import numpy as np
    import bench
    import rve_inputs as ri
    phi, _ = ri.octet(12, 0.2)
    lin, dt, cores = bench.j2_cpu_sample(phi.astype(np.float64), 110e9, 0.3, 70e6, 1.1e9, -2.5e-3, 7)
    assert lin == 7 and dt > 0 and cores >= 1


def test_step_stats_best_and_median():
    """best and median of the timed solves, and the rate of each"""
    import bench
    st = bench.step_stats([350.0, 340.0, 360.0, 345.0, 355.0], [4.0e9] * 5)
    assert st["n"] == 5 and st["best_ms"] == 340.0 and st["median_ms"] == 350.0
    assert abs(st["best_voxel_iters_per_s"] - 4.0e9 / 0.340) < 1.0
    assert abs(st["median_voxel_iters_per_s"] - 4.0e9 / 0.350) < 1.0
    assert bench.step_stats([], []) is None


def test_roofline_bytes_per_voxel():
    """the bench's algorithmic bytes: one MINRES iteration with FP32 fields
    reads five 6-component real fields (v_k, v_{k-1}, w_{k-1}, w_{k-2}, x,
    24 B each) and phi (4 B) and writes three (v_{k+1}, w_k, x): 196 B per
    voxel; a half spectrum of 6 complex64 per frequency holds (n/2+1)/n
    frequencies per voxel; the n2 passes read and write it once, the n3 pass
    also reads phi, the fused n1 pass reads 5 and writes 3 spectra plus x
    (read and written) on one step in three"""
    import bench
    assert bench.ITER_BYTES_PER_VOXEL == 5 * 24 + 4 + 3 * 24
    n = 256
    spec = 6 * 8 * (n // 2 + 1) / n
    kb = bench.kernel_bytes_per_voxel(n)
    assert abs(kb["x2_inv"] - 2 * spec) < 1e-9 and abs(kb["x2_fwd"] - 2 * spec) < 1e-9
    assert abs(kb["x3_c2r_law_energy_r2c"] - (2 * spec + 4)) < 1e-9
    assert abs(kb["x1_fwd_lanczos_inv"] - (5 + 3 + 2 / 3) * spec) < 1e-9
    # the figures quoted for 256^3: 48.4, 52.4, 209.6 and about 359 in all
    assert [round(kb[k], 1) for k in ("x2_inv", "x3_c2r_law_energy_r2c", "x1_fwd_lanczos_inv")] == [48.4, 52.4, 209.6]
    assert round(sum(kb.values())) == 359
