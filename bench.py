#!/usr/bin/env python
"""K-GRAPE hot-path benchmark: fidelity+gradient evaluations per second on GB300.

One step = one full evaluation (forward Krylov sweep over N slices, target overlap,
backward co-state sweep with the per-slice overlaps, gradient assembly) of the
L=20, N=400, m=20 XXZ workload, inputs resident in HBM.  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the CPU oracle (complex128 NumPy, one thread) on a bounded sample
of the same workload (one slice forward + one slice backward per step, extrapolated to
the N-slice evaluation).  Under torchrun each rank runs an independent replica
(the evaluation does not shard); value = evaluations of all ranks / slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
METRIC = "K-GRAPE fidelity+gradient evals/s (L=20,N=400) and HBM % of peak vs FP64"
UNIT = "evals/s"
DEFAULT_WORKLOAD = "xxz_L20_N400_m20"
FALLBACK_HBM_GBS = 6800.0


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--prec", choices=["c64", "c128", "ff"], default="c64",
                    help="ff (float-float vectors) runs on the subspace workloads (pe_...) only")
    ap.add_argument("--fp64-steps", type=int, default=2, help="timed steps of the plain FP64 (complex128) path")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--tile-bits", type=int, default=0)
    ap.add_argument("--ctas", type=int, default=0)
    ap.add_argument("--N", type=int, default=0, help="shorter pulse (profiling a small case); 0 = workload's N")
    ap.add_argument("--grad", choices=["centered", "zeroth", "exact", "taylor1", "taylor2"], default="centered",
                    help="gradient mode of the timed evaluations (the headline is the centred gradient; "
                         "taylor1/2 on subspace workloads only)")
    ap.add_argument("--reorth", action="store_true", help="full re-orthogonalisation of every Lanczos step")
    ap.add_argument("--phases", action="store_true",
                    help="print the headline loop's phase times (KG_FLAG_PHASE_TIMING, CTA 0) instead of a bench line")
    ap.add_argument("--batch", type=int, default=0,
                    help="pulses of a subspace workload (0: one per resident CTA of the subspace kernel)")
    return ap.parse_args()


def workload(name, N: int = 0):
    sys.path.insert(0, ROOT)
    import dataclasses

    from paper_2010_03598_gb300 import workloads as W
    w = W.WORKLOADS[name]
    if N:
        w = dataclasses.replace(w, N=N)
    return W, w


def alg_bytes(w, prec: str, ckpt: int = 0, grad: str = "centered") -> int:
    """Algorithmic HBM bytes of one evaluation: D-vector passes of the basis-storing Lanczos.

    Per slice and direction: Lanczos step k reads v_k and v_{k-1} (k >= 1) and writes
    v_{k+1} (k <= m-2): 3m-2 passes; the recombination reads m vectors and writes 1: m+1.
    The backward sweep reads psi_j once more for the gradient overlap; the target overlap
    reads 2 vectors.  P = N (2 (4m-1) + 1) + 2, plus N (4m-1) when checkpoints are
    recomputed, plus N (4 (m+1) + 2) for the exact gradient (two more recombinations per
    slice and direction, and the stored interior states read once).
    """
    s = 16 if prec == "c128" else 8
    P = w.N * (2 * (4 * w.m - 1) + 1) + 2
    if ckpt:
        P += w.N * (4 * w.m - 1)
    if grad == "exact":  # two more recombinations per slice each way, and the stored interior states
        P += w.N * (4 * (w.m + 1) + 2)
    return P * w.D * s


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


# Sources of the full-chain evaluation kernel and its host launch code (the subspace kernel,
# kg_sector.cu, is not part of the headline launch).
KERNEL_SOURCES = ("kg_abi.cu", "kg_device.cuh", "kg_eval.cu", "kg_internal.h", "kg_launch.h")


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2010_03598_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def err_vs_oracle(args, w, F, grad):
    """Relative error of a GPU result against the committed complex128 oracle values of the same
    seeded workload (tests/golden, written by the oracle alone): |dF|/F and ||dg||/||g||.  None if
    no golden covers this workload, pulse length and gradient mode."""
    if args.grad not in ("centered", "zeroth"):
        return None
    stem = f"oracle_{args.workload}" if w.N == 400 and args.workload == DEFAULT_WORKLOAD else None
    if stem is None:
        return None
    path = os.path.join(ROOT, "tests", "golden", stem + ".json")
    try:
        with open(path) as fh:
            gd = json.load(fh)
    except Exception:
        return None
    key_f, key_g = f"F_{args.grad}", f"grad_{args.grad}"
    if key_f not in gd or gd.get("N") != w.N:
        return None
    import numpy as np
    out = {"F": abs(F - gd[key_f]) / abs(gd[key_f]), "golden": f"tests/golden/{stem}.json"}
    if grad is not None and key_g in gd:
        g_ref = np.asarray(gd[key_g])
        out["grad"] = float(np.linalg.norm(np.asarray(grad) - g_ref) / np.linalg.norm(g_ref))
    return out


def short_pulse_golden(workload_name: str, grad: str):
    """A committed oracle golden of this workload on a shorter pulse (tests/golden), or None."""
    import glob
    for path in sorted(glob.glob(os.path.join(ROOT, "tests", "golden", "oracle_*.json"))):
        try:
            with open(path) as fh:
                gd = json.load(fh)
        except Exception:
            continue
        if gd.get("workload") == workload_name and f"F_{grad}" in gd:
            return path, gd
    return None


def err_vs_short_golden(A, W, w, args, dev):
    """Where no golden covers the timed pulse (the L = 24 chain: its oracle needs ~1.4 h of CPU for
    12 slices), evaluate the golden's shorter pulse once, untimed, with the same engine options (the
    checkpoint interval capped at the pulse's N - 1), and return the relative errors against it."""
    import dataclasses

    import numpy as np
    import torch
    found = short_pulse_golden(args.workload, args.grad)
    if found is None or args.grad not in ("centered", "zeroth"):
        return None
    path, gd = found
    n = int(gd["N"])
    ws = dataclasses.replace(w, N=n)
    u, psi0, f = W.instance(ws)
    ck = min(w.ckpt, max(n - 1, 0)) if w.ckpt > 0 else w.ckpt
    eng = A.KGrape(A.ChainSpec(w.L, w.Jxy, w.Jz), A.Options(n, w.dt, w.m, prec=args.prec, ckpt_every=ck,
                                                             grad=args.grad, reorth=args.reorth), device=dev)
    fid, grad = eng.evaluate(torch.tensor(u, device=dev), torch.tensor(psi0, device=dev),
                             torch.tensor(f, device=dev))
    eng.sync()
    F = float(fid.item())
    g = grad[:n].cpu().numpy()
    eng.close()
    ref = np.asarray(gd[f"grad_{args.grad}"])
    return {"F": abs(F - gd[f"F_{args.grad}"]) / abs(gd[f"F_{args.grad}"]),
            "grad": float(np.linalg.norm(g - ref) / np.linalg.norm(ref)),
            "golden": os.path.relpath(path, ROOT), "N": n, "ckpt_every": ck,
            "note": "a shorter pulse of the same workload, evaluated untimed with the timed options"}


def ncu_traffic(kernel_key: str):
    """DRAM bytes per launch from the committed ncu summary, if it matches this source."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        ent = d.get(kernel_key)
        if ent and ent.get("source_hash") == kernel_source_hash():
            return float(ent["dram_bytes_per_launch_full"])
    except Exception:
        pass
    return None


# ---------------------------------------------------------------- clocks during the timed region
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str | None):
        self.gpu_id = gpu_id
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
            if self.gpu_id:
                cmd.insert(1, f"--id={self.gpu_id}")
            self.proc = subprocess.Popen(cmd, stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        with open(self.path) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------- replicas (one process per GPU)
def replica_sync(world: int, device):
    """(barrier, max_over_ranks) for independent replicas: the evaluation does not shard, so the
    only collectives are the barrier around the timed region and the slowest rank's time."""
    import torch
    import torch.distributed as dist

    def barrier():
        if world > 1:
            dist.barrier()

    def max_over_ranks(x: float) -> float:
        if world == 1:
            return x
        t = torch.tensor([x], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    return barrier, max_over_ranks


def job_throughput(units_per_rank: int, seconds_this_rank: float, world: int, max_over_ranks):
    """Whole-job value: every rank processed units_per_rank; the job took the slowest rank's time."""
    t = max_over_ranks(seconds_this_rank)
    return units_per_rank * world / t, t


# ---------------------------------------------------------------- CPU oracle sample
ORACLE_SNIPPET = r"""
import json, sys, time
sys.path.insert(0, {root!r})
import numpy as np
import oracle
from paper_2010_03598_gb300 import workloads as W
w = W.WORKLOADS[{name!r}]
u, psi0, f = W.instance(w, N={slices})
ch = oracle.Chain(w.L, w.Jxy, w.Jz)
t0 = time.perf_counter()
oracle.segment_forward_backward(ch, u, w.dt, w.m, psi0, f)
dt = time.perf_counter() - t0
print(json.dumps(dict(seconds=dt, slices={slices})))
"""

THREAD_ENV = {"OMP_NUM_THREADS": "1", "OPENBLAS_NUM_THREADS": "1", "MKL_NUM_THREADS": "1"}


def cpu_baseline(wname: str, w, slices: int = 1):
    env = dict(os.environ, **THREAD_ENV)
    code = ORACLE_SNIPPET.format(root=ROOT, name=wname, slices=slices)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=900)
    if r.returncode != 0:
        return {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle", "error": r.stderr[-300:]}
    d = json.loads(r.stdout.strip().splitlines()[-1])
    per_eval = d["seconds"] * w.N / slices
    return {"value": 1.0 / per_eval, "unit": UNIT, "cores": 1, "host_cores": os.cpu_count(), "kind": "oracle",
            "sample": f"{slices} slice(s) forward + backward of the {wname} workload "
                      f"({d['seconds']:.2f} s), extrapolated x{w.N // slices} to one evaluation; "
                      "NumPy complex128, 1 thread (OMP/OpenBLAS/MKL = 1)"}


# ---------------------------------------------------------------- reference arm (the oracle)
def run_reference(args):
    for k, v in THREAD_ENV.items():
        os.environ[k] = v
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    W, w = workload(args.workload, args.N)
    import oracle
    u, psi0, f = W.instance(w, N=1)
    ch = oracle.Chain(w.L, w.Jxy, w.Jz)
    for _ in range(args.warmup):
        oracle.segment_forward_backward(ch, u, w.dt, w.m, psi0, f)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.segment_forward_backward(ch, u, w.dt, w.m, psi0, f)
        times.append(time.perf_counter() - t0)
    step_s = statistics.mean(times)
    per_eval = step_s * w.N
    value = 1.0 / per_eval
    out = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_s * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "c128", "data": "synthetic",
        "config": dict(config_block(w, args.workload, "c128"), grad=args.grad, reorth=bool(args.reorth)),
        "step": f"1 slice forward + 1 slice backward of the {w.N}-slice evaluation",
        "extrapolated_ms_per_eval": per_eval * 1e3,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "host_cores": os.cpu_count(), "kind": "oracle",
                         "sample": f"each step = 1 slice forward + 1 slice backward of {args.workload} "
                                   f"(mean {step_s:.2f} s), extrapolated x{w.N} to one evaluation; NumPy complex128, "
                                   "1 thread"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out))


def config_block(w, name, prec):
    return {"workload": name, "L": w.L, "D": w.D, "N": w.N, "m": w.m, "dt": w.dt, "delta": w.delta, "J": w.J,
            "ckpt_every": w.ckpt,
            "hc": "Sx on site 1", "psi0": "Neel", "target": "seeded Gaussian, normalised", "prec": prec,
            "l2": "flushed between timed steps (512 MiB write); per-step working set > L2",
            "parallelism": "replicas (one independent evaluation per GPU)"}


# ---------------------------------------------------------------- our arm
def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    sys.path.insert(0, ROOT)
    from paper_2010_03598_gb300 import api as A
    W, w = workload(args.workload, args.N)

    barrier, max_over_ranks = replica_sync(world, dev)

    u, psi0, f = W.instance(w)
    ut = torch.tensor(u, device=dev)
    pt = torch.tensor(psi0, device=dev)
    ft = torch.tensor(f, device=dev)
    chain = A.ChainSpec(w.L, w.Jxy, w.Jz)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def timed(prec, steps, warmup):
        eng = A.KGrape(chain, A.Options(w.N, w.dt, w.m, prec=prec, tile_bits=args.tile_bits, ctas=args.ctas,
                                        ckpt_every=w.ckpt, grad=args.grad, reorth=args.reorth), device=dev)
        for _ in range(warmup):
            eng.evaluate(ut, pt, ft)
        rep = eng.sync()
        torch.cuda.synchronize(dev)
        barrier()
        torch.cuda.synchronize(dev)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        t_wall = time.perf_counter()
        for e0, e1 in ev:
            flush.fill_(1)                     # evict L2 between steps (outside the events)
            e0.record(stream)
            eng.evaluate(ut, pt, ft)
            e1.record(stream)
        torch.cuda.synchronize(dev)
        t_wall = time.perf_counter() - t_wall
        barrier()
        rep = eng.sync()
        ms = [e0.elapsed_time(e1) for e0, e1 in ev]
        fid = float(eng.fid.item())
        grad = eng.grad[: w.N].cpu().numpy().copy() if args.grad != "none" else None
        eng.close()
        return ms, rep, fid, t_wall, grad

    gpu_id = None
    try:
        props = torch.cuda.get_device_properties(dev)
        gpu_id = f"{props.pci_domain_id:08X}:{props.pci_bus_id:02X}:{props.pci_device_id:02X}.0"
    except Exception:
        gpu_id = None

    # --- headline path (timed region sampled for clocks)
    sampler = ClockSampler(gpu_id)
    sampler.start()
    ms, rep, fid, wall, grad = timed(args.prec, args.steps, args.warmup)
    clocks = sampler.stop()
    value, total_s = job_throughput(args.steps, sum(ms) / 1e3, world, max_over_ranks)
    ms_per_step = total_s * 1e3 / args.steps
    hbm, peak_kind = measured_peaks()
    per_launch_s = statistics.mean(ms) / 1e3
    ab = alg_bytes(w, args.prec, w.ckpt, args.grad)
    achieved = ab / per_launch_s / 1e9
    kernel_key = f"kg_eval_kernel<{'float2' if args.prec == 'c64' else 'double2'}>@{args.workload}"
    roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                "traffic": ncu_traffic(kernel_key), "peak_kind": peak_kind,
                "algorithmic_bytes_per_launch": ab, "kernel": kernel_key.split("@")[0],
                "launch_ms": statistics.mean(ms)}

    # --- plain FP64 path, same workload
    fp64 = None
    if args.fp64_steps > 0 and args.prec != "c128":
        ms64, rep64, fid64, _, grad64 = timed("c128", args.fp64_steps, 1)
        t64 = max_over_ranks(sum(ms64) / 1e3)
        a64 = alg_bytes(w, "c128", w.ckpt) / (statistics.mean(ms64) / 1e3) / 1e9
        fp64 = {"value": args.fp64_steps * world / t64, "unit": UNIT, "ms_per_step": t64 * 1e3 / args.fp64_steps,
                "steps": args.fp64_steps, "hbm_gbs_algorithmic": a64, "hbm_frac": a64 / hbm,
                "speedup_of_headline": value / (args.fp64_steps * world / t64),
                "rel_diff_F_vs_headline": abs(fid - fid64) / abs(fid64),
                "err_vs_oracle": err_vs_oracle(args, w, fid64, grad64)}

    # --- end to end through the C ABI with host buffers (pinned), copies inside the timed region
    e2e = None
    if args.e2e_steps > 0:
        e2e = run_e2e(A, chain, w, args, dev, u, psi0, f, barrier, max_over_ranks, world)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args.workload, w)
        if args.grad != "centered" and cpu.get("sample"):
            cpu["sample"] += "; the oracle's centred gradient, not the timed gradient mode"
    err = err_vs_oracle(args, w, fid, grad)
    if err is None and rank == 0 and args.N == 0:  # the workload's own pulse length only
        err = err_vs_short_golden(A, W, w, args, dev)
    emit(rank, world, args, w, value, ms_per_step, roofline, cpu, e2e, clocks, fp64, rep, fid, wall, err)
    if world > 1:
        dist.destroy_process_group()


def run_e2e(A, chain, w, args, dev, u, psi0, f, barrier, max_over_ranks, world):
    import torch
    eng = A.KGrape(chain, A.Options(w.N, w.dt, w.m, prec=args.prec, host_staging=True, tile_bits=args.tile_bits,
                                    ctas=args.ctas, ckpt_every=w.ckpt, grad=args.grad, reorth=args.reorth),
                   device=dev)
    uh = torch.tensor(u).pin_memory()
    ph = torch.tensor(psi0).pin_memory()
    fh = torch.tensor(f).pin_memory()
    fid_h = torch.zeros(1, dtype=torch.float64).pin_memory()
    grad_h = torch.zeros(w.N, dtype=torch.float64).pin_memory()
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    eng.evaluate_host(uh, ph, fh, fid_h, grad_h)
    torch.cuda.synchronize(dev)
    barrier()
    te_local = 0.0
    for _ in range(args.e2e_steps):
        flush.fill_(1)  # evict L2 between steps, as the device-timed leg does (outside the timed call)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        eng.evaluate_host(uh, ph, fh, fid_h, grad_h)  # returns after the results are on the host
        te_local += time.perf_counter() - t0
    te = max_over_ranks(te_local)
    eng.close()
    return {"value": args.e2e_steps * world / te, "unit": UNIT,
            "h2d_bytes_per_step": int(uh.numel() * 8 + ph.numel() * 16 + fh.numel() * 16),
            "d2h_bytes_per_step": int(8 + grad_h.numel() * 8), "api": "kg_evaluate_host (pinned host buffers)",
            "l2": "flushed between steps (512 MiB write, outside the timed call)"}


def emit(rank, world, args, w, value, ms_per_step, roofline, cpu, e2e, clocks, fp64, rep, fid, wall, err=None):
    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "c64+f64" if args.prec == "c64" else "c128", "data": "synthetic",
            "config": dict(config_block(w, args.workload, args.prec), grad=args.grad, reorth=bool(args.reorth)),
            "roofline": roofline, "cpu_baseline": cpu,
            "e2e": e2e, "clocks": clocks, "gpu_launches": args.steps, "fp64_path": fp64,
            "report": {k: rep[k] for k in ("krylov_err_max", "norm_final", "breakdowns", "ctas", "tile_bits",
                                           "threads")},
            "F": fid, "err_vs_oracle": err, "wall_s_timed": wall,
        }
        print(json.dumps(out))


BATCH_WORKLOAD = "batch256"
BATCH_METRIC = "K-GRAPE batched fidelity+gradient evals/s (256 pulses, L 10..16, N=200, m=16)"


def run_batch(args):
    """The batched workload: 256 independent pulses in one graph-captured cooperative launch."""
    import torch

    sys.path.insert(0, ROOT)
    from paper_2010_03598_gb300 import api as A
    from paper_2010_03598_gb300 import tune
    from paper_2010_03598_gb300 import workloads as W

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    inst = W.batch_instances()
    N, dt, m = W.BATCH_N, W.BATCH_DT, W.BATCH_M
    chains = [A.ChainSpec(d["L"], 1.0, d["delta"]) for d in inst]
    u = [torch.tensor(d["u"], device=dev) for d in inst]
    psi0 = [torch.tensor(d["psi0"], device=dev) for d in inst]
    target = [torch.tensor(d["target"], device=dev) for d in inst]
    opts = A.Options(N, dt, m, prec="c64")
    best = tune.tune_batch(chains, opts, u, psi0, target, device=dev)
    stream = torch.cuda.Stream(dev)
    b = A.KGrapeBatch(chains, opts, u, psi0, target, device=dev, stream=stream, ctas=best["ctas"],
                      tiles_per_cta=best["tiles_per_cta"])
    for _ in range(args.warmup):
        b.launch()
    b.sync()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        b.launch()
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    ms = []
    sampler = ClockSampler(None)
    sampler.start()
    for _ in range(args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(1)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            g.replay()
            e1.record(stream)
        torch.cuda.synchronize(dev)
        ms.append(e0.elapsed_time(e1))
    clocks = sampler.stop()
    b.sync()
    B = len(inst)
    t = sum(ms) / 1e3
    value = B * args.steps / t
    P = N * (2 * (4 * m - 1) + 1) + 2
    ab = sum(P * (1 << d["L"]) * 8 for d in inst)
    hbm, kind = measured_peaks()
    achieved = ab / (statistics.mean(ms) / 1e3) / 1e9
    out = {"metric": BATCH_METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": statistics.mean(ms), "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "c64+f64", "data": "synthetic",
           "config": {"workload": BATCH_WORKLOAD, "pulses": B, "L": "U{10..16}", "N": N, "m": m, "dt": dt,
                      "delta": "U(0,2)", "schedule": {k: best[k] for k in ("ctas", "tiles_per_cta")},
                      "launch": "one cooperative kernel per batch, replayed from a CUDA graph",
                      "l2": "flushed between timed replays (512 MiB write)"},
           "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                        "traffic": None, "peak_kind": kind, "algorithmic_bytes_per_launch": ab,
                        "kernel": "kg_batch_kernel"},
           "tuning": best.get("trials"), "clocks": clocks, "gpu_launches": args.steps}
    print(json.dumps(out))
    b.close()


SECTOR_METRIC = "K-GRAPE fidelity+gradient evals/s in a parity-excitation subspace (Sec. 3.1 task, M = 4D)"

SECTOR_ORACLE_SNIPPET = r"""
import json, sys, time
sys.path.insert(0, {root!r})
import oracle, oracle.sector as S
from paper_2010_03598_gb300 import workloads as W
w = W.SECTOR_WORKLOADS[{name!r}]
c = S.paper_chain(w.L, w.K, w.parity)
U, psi0, f = W.sector_instance(w, c.D, batch=1, N={slices})
t0 = time.perf_counter()
oracle.evaluate(c, U[0], w.dt, w.m, psi0, f, "centered")
print(json.dumps(dict(seconds=time.perf_counter() - t0, slices={slices})))
"""


def resident_pulses(A, spec, w, D, prec, dev) -> int:
    """Pulses that fill every CTA the subspace kernel keeps resident (one pulse per CTA): the grid a
    probe engine (two slices, more pulses than fit) chooses on this device."""
    import torch

    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    probe = A.KGrapeSector(spec, A.Options(2, w.dt, w.m, prec=prec, grad="none"), B=8 * sms)
    z = torch.zeros(8 * sms, 2, dtype=torch.float64, device=dev)
    e = torch.zeros(D, dtype=torch.complex128, device=dev)
    e[0] = 1.0
    probe.evaluate(z, e, e)
    ctas = int(probe.sync()["ctas"])
    probe.close()
    return ctas


def run_sector(args):
    """Sec. 3.1-3.2's own setting: B pulses of the e_1 -> e_D task in one PE subspace, one CTA per pulse."""
    import torch

    sys.path.insert(0, ROOT)
    from paper_2010_03598_gb300 import api as A
    from paper_2010_03598_gb300 import workloads as W

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    w = W.SECTOR_WORKLOADS[args.workload]
    spec = A.SectorSpec(w.L, w.K, w.parity, Jxy=2.0 * w.J, Jz=2.0 * w.J * w.alpha_z, hc_amp=w.J)
    D = A.sector_dim(spec)
    B = args.batch if args.batch > 0 else resident_pulses(A, spec, w, D, args.prec, dev)
    U, psi0, f = W.sector_instance(w, D, batch=B)
    N = U.shape[1]
    ut, pt, ft = torch.tensor(U, device=dev), torch.tensor(psi0, device=dev), torch.tensor(f, device=dev)
    eng = A.KGrapeSector(spec, A.Options(N, w.dt, w.m, prec=args.prec, grad=args.grad), B=B)
    stream = torch.cuda.current_stream(dev)
    for _ in range(args.warmup):
        eng.evaluate(ut, pt, ft)
    rep = eng.sync()
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    sampler = ClockSampler(None)
    sampler.start()
    torch.cuda.synchronize(dev)
    t_wall = time.perf_counter()
    for e0, e1 in ev:
        flush.fill_(1)
        e0.record(stream)
        eng.evaluate(ut, pt, ft)
        e1.record(stream)
    torch.cuda.synchronize(dev)
    t_wall = time.perf_counter() - t_wall
    clocks = sampler.stop()
    rep = eng.sync()
    ms = [e0.elapsed_time(e1) for e0, e1 in ev]
    value = B * args.steps / (sum(ms) / 1e3)
    # algorithmic bytes as for the full chain (D-vector passes of the basis-storing Lanczos with the
    # centred gradient), per pulse; the other gradient modes are timed against the same count
    s = 8 if args.prec == "c64" else 16
    ab = B * (N * (2 * (4 * w.m - 1) + 1) + 2) * D * s
    hbm, kind = measured_peaks()
    achieved = ab / (statistics.mean(ms) / 1e3) / 1e9
    fid0 = float(eng.fid[0].item())
    # end to end: pinned host controls in, F and gradients out, inside the timed region
    e2e = None
    if args.e2e_steps > 0:
        uh = torch.tensor(U).pin_memory()
        fid_h = torch.zeros(B, dtype=torch.float64).pin_memory()
        grad_h = torch.zeros(B, N, dtype=torch.float64).pin_memory()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            ut.copy_(uh, non_blocking=True)
            fid, grad = eng.evaluate(ut, pt, ft)
            fid_h.copy_(fid, non_blocking=True)
            grad_h.copy_(grad, non_blocking=True)
            eng.sync()
        te = time.perf_counter() - t0
        e2e = {"value": B * args.e2e_steps / te, "unit": UNIT, "h2d_bytes_per_step": int(uh.numel() * 8),
               "d2h_bytes_per_step": int(fid_h.numel() * 8 + grad_h.numel() * 8),
               "api": "KGrapeSector.evaluate + sync, controls copied in from pinned host memory"}
    cpu = None
    if not args.no_cpu_baseline:
        sl = min(N, 200)
        env = dict(os.environ, **THREAD_ENV)
        r = subprocess.run([sys.executable, "-c", SECTOR_ORACLE_SNIPPET.format(root=ROOT, name=args.workload,
                                                                               slices=sl)],
                           capture_output=True, text=True, env=env, timeout=900)
        if r.returncode == 0:
            d = json.loads(r.stdout.strip().splitlines()[-1])
            per = d["seconds"] * N / sl
            cpu = {"value": 1.0 / per, "unit": UNIT, "cores": 1, "kind": "oracle",
                   "sample": f"one pulse of {sl} slices forward + backward ({d['seconds']:.2f} s), extrapolated "
                             f"x{N / sl:.1f} to the M = 4D = {N}-slice pulse; NumPy/SciPy complex128, 1 thread"}
        else:
            cpu = {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle", "error": r.stderr[-300:]}
    out = {"metric": SECTOR_METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": statistics.mean(ms), "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": {"c64": "c64+f64", "c128": "c128", "ff": "ff32x2+f64"}[args.prec],
           "data": "synthetic",
           "config": {"workload": args.workload, "L": w.L, "K": w.K, "prec": args.prec, "parity": w.parity, "D": D, "N": N, "m": w.m,
                      "dt": w.dt, "pulses": B, "task": "e_1 -> e_D", "J": w.J, "alpha_z": w.alpha_z,
                      "grad": args.grad,
                      "hc": "(J/2)(sigma^z_1 + sigma^z_L)", "u": "U(-1,1)",
                      "l2": "flushed between timed steps (512 MiB write); per-step working set > L2",
                      "launch": "one CTA per pulse, state in shared memory"},
           "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                        "traffic": None, "peak_kind": kind, "algorithmic_bytes_per_launch": ab,
                        "kernel": "kg_sector_kernel",
                        "note": "the D-vector passes are served from shared memory; the kernel is bound by "
                                "block-barrier and FP64 latency, not by HBM"},
           "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks, "gpu_launches": args.steps,
           "report": {k: rep[k] for k in ("krylov_err_max", "breakdowns", "ctas", "threads")},
           "F_pulse0": fid0, "wall_s_timed": t_wall}
    print(json.dumps(out))
    eng.close()


def run_phases(args):
    """Phase times of the complex64 evaluation (clock64 marks of CTA 0's thread 0, KG_FLAG_PHASE_TIMING):
    per Lanczos step and per slice, in microseconds at the SM clock read from nvidia-smi (2070 MHz if
    unavailable).  A diagnostic: the marks add a little time, and the numbers are not a bench value."""
    import torch

    sys.path.insert(0, ROOT)
    from paper_2010_03598_gb300 import api as A
    W, w = workload(args.workload, args.N or 20)
    dev = torch.device("cuda", 0)
    u, psi0, f = W.instance(w)
    eng = A.KGrape(A.ChainSpec(w.L, w.Jxy, w.Jz), A.Options(w.N, w.dt, w.m, prec="c64", phase_timing=True),
                   device=dev)
    ut, pt, ft = (torch.tensor(x, device=dev) for x in (u, psi0, f))
    for _ in range(2):
        eng.evaluate(ut, pt, ft)
    pc = eng.sync()["phase_cycles"]
    eng.close()
    mhz = 2070.0
    try:
        r = subprocess.run(["nvidia-smi", "--query-gpu=clocks.sm", "--format=csv,noheader,nounits", "-i", "0"],
                           capture_output=True, text=True, timeout=20)
        mhz = float(r.stdout.strip().splitlines()[0]) or mhz
    except Exception:
        pass
    us = [c / mhz for c in pc]
    steps, slices = 2 * w.N * w.m, 2 * w.N
    print(json.dumps({"workload": args.workload, "N": w.N, "sm_mhz": mhz, "total_us": us[7],
                      "per_step_us": {"partner blocks": us[0] / steps, "update": us[1] / steps,
                                      "hand-over, stencil, group wait": us[2] / steps,
                                      "wait for the scalars": us[3] / steps},
                      "per_slice_us": {"last barrier, T, exponential, coefficients": us[4] / slices,
                                       "recombination, store, end-of-slice reduction": us[5] / slices}}))


def main():
    args = parse_args()
    if args.phases:
        run_phases(args)
        return
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == BATCH_WORKLOAD:
        run_batch(args)
    elif args.workload.startswith("pe_"):
        run_sector(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
