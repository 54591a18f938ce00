"""Schedule autotuner for batched evaluations.

Times candidate launch schedules (CTAs of the launch, tiles per CTA, i.e. how many CTAs a
problem's group gets) of a batch on the current GPU through the C ABI and caches the
fastest per (GPU name, batch signature) in a JSON file (``$KG_TUNE_CACHE``, default
``~/.cache/kgrape_tune.json``).  Every candidate computes the same results; only the time
differs.
"""
from __future__ import annotations

import hashlib
import json
import os

import torch

from . import api

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "kgrape_tune.json")


def signature(chains, opts: api.Options) -> str:
    h = hashlib.sha256()
    h.update(repr((opts.N, opts.m, opts.dt, opts.prec, opts.grad, opts.ckpt_every)).encode())
    for c in chains:
        h.update(repr((c.L, c.hc_kind, c.hc_site, c.hc_mask)).encode())
    return h.hexdigest()[:16]


def _load(path):
    try:
        with open(path) as fh:
            return json.load(fh)
    except Exception:
        return {}


def candidates(device) -> list[dict]:
    sms = torch.cuda.get_device_properties(device).multi_processor_count
    out = []
    for ctas in sorted({sms, (sms // 8) * 8, sms // 2}, reverse=True):
        for tpc in (2, 1):
            out.append(dict(ctas=ctas, tiles_per_cta=tpc))
    return out


def tune_batch(chains, opts: api.Options, u, psi0, target, device=None, repeats: int = 2,
               cache_path: str | None = None, force: bool = False) -> dict:
    """Return the fastest schedule {ctas, tiles_per_cta, ms} for this batch (cached)."""
    device = torch.device("cuda", torch.cuda.current_device() if device is None else torch.device(device).index or 0)
    path = cache_path or os.environ.get("KG_TUNE_CACHE", DEFAULT_CACHE)
    key = f"{torch.cuda.get_device_name(device)}|{signature(chains, opts)}"
    cache = _load(path)
    if key in cache and not force:
        return cache[key]
    best = None
    trials = []
    for cand in candidates(device):
        b = api.KGrapeBatch(chains, opts, u, psi0, target, device=device, **cand)
        b.launch()
        b.sync()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(b.stream)
        for _ in range(repeats):
            b.launch()
        e1.record(b.stream)
        b.sync()
        ms = e0.elapsed_time(e1) / repeats
        b.close()
        trials.append(dict(cand, ms=ms))
        if best is None or ms < best["ms"]:
            best = dict(cand, ms=ms)
    best = dict(best, trials=trials)
    cache[key] = best
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        with open(path, "w") as fh:
            json.dump(cache, fh, indent=1)
    except OSError:
        pass
    return best
