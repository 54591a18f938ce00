"""Write the oracle's expected values for the GPU parity tests.

Every value stored here is computed by ``oracle/`` alone (complex128 CPU oracle) on the
seeded inputs of ``paper_2010_03598_gb300.workloads``; nothing comes from the CUDA
path.  Run from the repository root:  python tests/golden/make_golden.py
"""
from __future__ import annotations

import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_2010_03598_gb300 import workloads as W  # noqa: E402

CASES = [
    # (file stem, workload, N override, gradient modes)
    ("oracle_xxz_L8_N64_m12", "xxz_L8_N64_m12", None, ("centered", "zeroth")),
    ("oracle_xxz_L16_N200_m20", "xxz_L16_N200_m20", None, ("centered",)),
    ("oracle_xxz_L20_N2_m20", "xxz_L20_N400_m20", 2, ("centered", "zeroth")),
    # the benchmarked pulse in full (about half an hour of one CPU core)
    ("oracle_xxz_L20_N400_m20", "xxz_L20_N400_m20", None, ("centered",)),
    # the checkpointed chain at its full size, on a 12-slice pulse (a few GB of host memory)
    ("oracle_xxz_L24_N12_m24", "xxz_L24_N400_m24_ckpt20", 12, ("centered",)),
]


def run(stem, wname, N, modes):
    w = W.WORKLOADS[wname]
    u, psi0, f = W.instance(w, N=N)
    ch = oracle.Chain(w.L, w.Jxy, w.Jz)
    out = dict(workload=wname, L=w.L, N=len(u), dt=w.dt, m=w.m, Jxy=w.Jxy, Jz=w.Jz, seed=w.seed,
               source="oracle/ (complex128, full CGS2 Lanczos, eigh), tests/golden/make_golden.py")
    t0 = time.time()
    for mode in modes:
        F, g, d = oracle.evaluate(ch, u, w.dt, w.m, psi0, f, mode)
        out[f"F_{mode}"] = F
        out[f"grad_{mode}"] = [float(x) for x in g]
        out["beta"] = [d["beta"].real, d["beta"].imag]
        out["G"] = [float(x) for x in d["G"]]
        out["krylov_err_max"] = max(d["err_fwd"], d["err_bwd"])
        out["norm_final"] = float(np.linalg.norm(d["psi_N"]))
    out["F"] = out[f"F_{modes[0]}"]
    out["seconds"] = time.time() - t0
    with open(os.path.join(HERE, stem + ".json"), "w") as fh:
        json.dump(out, fh, indent=1, sort_keys=True)
    print(f"{stem}: F={out['F']!r} ({out['seconds']:.1f}s)")


if __name__ == "__main__":
    only = set(sys.argv[1:])
    for case in CASES:
        if not only or case[0] in only:
            run(*case)
