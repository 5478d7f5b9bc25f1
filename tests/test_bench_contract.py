"""CPU checks of bench.py's contract: the reference arm's JSON line, the
multi-rank timing aggregation (gloo, world size 2), and rank > 0 silence."""
import json
import os
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_line():
    env = dict(os.environ, OMP_NUM_THREADS="2")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "2",
                        "--warmup", "1"], capture_output=True, text=True, env=env, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "MLUPS" and d["value"] > 0
    assert d["higher_is_better"] is True and d["n_gpus"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]


def test_reference_arm_other_ranks_are_silent():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "1"], capture_output=True, text=True, env=env, timeout=300, cwd=ROOT)
    assert r.returncode == 0 and r.stdout.strip() == ""


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import bench

    dist = bench.init_dist(world, "gloo")
    local_ms = 10.0 + 5.0 * rank  # rank 1 is the slow one
    bench.barrier(world)
    ms_max = bench.max_over_ranks(local_ms, world)
    out[rank] = (ms_max, bench.aggregate(1000, 10, ms_max, world))
    dist.destroy_process_group()


def test_multi_rank_timing_takes_the_slowest_rank():
    port = 29500 + os.getpid() % 1000
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    for rank in (0, 1):
        ms_max, value = res[rank]
        assert ms_max == 15.0
        # whole-job throughput: both replicas' updates over the slowest time
        assert value == pytest.approx(2 * 1000 * 10 / 15e-3 / 1e6)


def test_kernel_fraction_arithmetic():
    """kernel_frac: bytes per cell x cells / launch time / peak (the adjoint
    kernel of the sphere: 456 B x 2e6 cells in 0.2230 ms = 4.09 TB/s, 0.610 of
    6701.5 GB/s)."""
    import bench

    class Lattice:
        N = 2_000_000

    assert abs(bench.kernel_frac(Lattice, 0.2230, 456, 6701.5) - 912e6 / 0.2230e-3 / 6701.5e9) < 1e-12
    assert abs(bench.kernel_frac(Lattice, 0.2230, 456, 6701.5) - 0.6103) < 1e-4
