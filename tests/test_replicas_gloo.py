"""The multi-GPU path of the benchmark is replicas only (the evaluation does not shard): the
collectives are a barrier and the slowest rank's time.  Two gloo ranks on the CPU exercise that
host logic; the reference arm runs on rank 0 alone."""
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    barrier, max_over_ranks = bench.replica_sync(world, torch.device("cpu"))
    barrier()
    # rank r took (r + 1) seconds for its 5 evaluations: the job took 2 s for 10 evaluations
    value, t = bench.job_throughput(5, float(rank + 1), world, max_over_ranks)
    barrier()
    out[rank] = (value, t)
    dist.destroy_process_group()


def test_two_gloo_replicas_report_the_slowest_rank():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    assert res[0] == res[1] == (5.0, 2.0)  # 10 evaluations / 2 s, identical on both ranks


def test_single_process_needs_no_collective():
    sys.path.insert(0, ROOT)
    import bench

    barrier, max_over_ranks = bench.replica_sync(1, None)
    barrier()
    assert bench.job_throughput(4, 2.0, 1, max_over_ranks) == (2.0, 2.0)


def test_reference_arm_prints_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, env=env, timeout=300, cwd=ROOT)
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_algorithmic_bytes_of_the_benchmark_lines():
    # D-vector passes of the basis-storing Lanczos, P = N (2 (4m - 1) + 1) + 2 (+ N (4m - 1) with
    # checkpoint recompute): 533.5 GB for L=20, N=400, m=20 in complex64, twice that in complex128,
    # 15.35 TB for L=24, N=400, m=24 with checkpoints every 20
    sys.path.insert(0, ROOT)
    import bench
    from paper_2010_03598_gb300 import workloads as W

    w20 = W.WORKLOADS["xxz_L20_N400_m20"]
    assert bench.alg_bytes(w20, "c64") == (400 * 159 + 2) * (1 << 20) * 8
    assert abs(bench.alg_bytes(w20, "c64") / 1e9 - 533.5) < 0.1
    assert bench.alg_bytes(w20, "c128") == 2 * bench.alg_bytes(w20, "c64")
    w24 = W.WORKLOADS["xxz_L24_N400_m24_ckpt20"]
    assert abs(bench.alg_bytes(w24, "c64", w24.ckpt) / 1e12 - 15.35) < 0.01
    # the exact gradient adds two recombinations per slice and direction and the stored interior states
    assert bench.alg_bytes(w20, "c64", 0, "exact") - bench.alg_bytes(w20, "c64") == 400 * (4 * 21 + 2) * (1 << 20) * 8
