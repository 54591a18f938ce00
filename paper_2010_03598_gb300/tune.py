"""Schedule autotuner: times candidate launch schedules through the C ABI on the current GPU and
caches the fastest in a JSON file (``$KG_TUNE_CACHE``, default ``~/.cache/kgrape_tune.json``).

Three searches, each keyed by (GPU name, kind, the problem's size, m, precision, gradient mode):

* ``tune_single``: tile size x CTAs of a single-problem engine (``Options.tile_bits``, ``ctas``);
  the tile size decides the loop (resident pairs of 4096-amplitude tiles, resident smaller
  tiles, streaming) and the CTAs how the tiles are dealt.
* ``tune_sector``: threads per CTA of the parity-excitation subspace kernel
  (``SectorSpec.block_threads``) and its grid (``Options.ctas``: CTAs, i.e. pulses in flight).
* ``tune_batch``: CTAs of the batched launch and tiles per CTA.

Every candidate computes the same quantity; schedules that change the tiling sum in another
order, so results agree to rounding (and bitwise where only the grid of the same loop changes).
A candidate the library refuses is skipped.  ``timer`` replaces the GPU timing (it receives the
candidate and returns milliseconds), which lets the search and the cache be checked without a GPU.
"""
from __future__ import annotations

import dataclasses
import hashlib
import json
import os

from . import _abi, api

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "kgrape_tune.json")


def _load(path):
    try:
        with open(path) as fh:
            return json.load(fh)
    except Exception:
        return {}


def _store(path, cache):
    try:
        os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
        with open(path, "w") as fh:
            json.dump(cache, fh, indent=1, sort_keys=True)
    except OSError:
        pass


def cache_key(gpu: str, kind: str, **size) -> str:
    """`gpu|kind|k=v,...` over the sorted size fields (e.g. L, m, prec, grad)."""
    return f"{gpu}|{kind}|" + ",".join(f"{k}={size[k]}" for k in sorted(size))


def search(key: str, candidates: list[dict], measure, cache_path: str | None = None, force: bool = False) -> dict:
    """The fastest candidate by `measure(cand) -> ms` (cached under `key`): {..cand, ms, trials}."""
    path = cache_path or os.environ.get("KG_TUNE_CACHE", DEFAULT_CACHE)
    cache = _load(path)
    if key in cache and not force:
        return cache[key]
    best, trials = None, []
    for cand in candidates:
        try:
            ms = float(measure(cand))
        except (_abi.KGrapeError, RuntimeError, ValueError):
            trials.append(dict(cand, ms=None))
            continue
        trials.append(dict(cand, ms=ms))
        if best is None or ms < best["ms"]:
            best = dict(cand, ms=ms)
    if best is None:
        raise RuntimeError(f"no schedule of {key} could run")
    best = dict(best, trials=trials)
    cache[key] = best
    _store(path, cache)
    return best


def _gpu(device):
    import torch
    dev = torch.device("cuda", torch.cuda.current_device() if device is None else torch.device(device).index or 0)
    props = torch.cuda.get_device_properties(dev)
    return dev, props.name, props.multi_processor_count


def _time_events(run, repeats: int, stream=None) -> float:
    import torch
    run()  # warm-up (and the first call's set-up)
    torch.cuda.synchronize()
    s = stream if stream is not None else torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(repeats):
        run()
    e1.record(s)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / repeats


# ---------------------------------------------------------------- single problem
def single_candidates(L: int, prec: str, sms: int) -> list[dict]:
    """Tile sizes (amplitudes 2^t) x CTAs: the library's default first, then the resident pairs
    of 4096-amplitude tiles (complex64), smaller tiles and the streaming loops on every SM."""
    tmax = 12 if prec == "c64" else 11
    out = [dict(tile_bits=0, ctas=0)]
    for t in range(min(tmax, L), max(min(tmax, L) - 3, 0), -1):
        ntiles = 1 << (L - t)
        grids = {min(ntiles, sms), min(ntiles, (sms // 8) * 8)}
        if ntiles // 2 <= sms:  # two tiles per CTA, all co-resident
            grids.add(max(1, ntiles // 2))
        for c in sorted(grids, reverse=True):
            cand = dict(tile_bits=t, ctas=c)
            if cand not in out:
                out.append(cand)
    return out


def tune_single(chain: api.ChainSpec, opts: api.Options, u, psi0, target, device=None, repeats: int = 2,
                cache_path: str | None = None, force: bool = False, timer=None, gpu: str | None = None,
                sms: int | None = None) -> dict:
    """Fastest (tile_bits, ctas) for single evaluations of this chain size and options."""
    if timer is None:
        dev, gpu, sms = _gpu(device)

        def timer(cand):
            eng = api.KGrape(chain, dataclasses.replace(opts, **cand), device=dev)
            try:
                def run():
                    eng.evaluate(u, psi0, target)
                ms = _time_events(run, repeats, eng.stream)
                eng.sync()
                return ms
            finally:
                eng.close()
    key = cache_key(gpu or "gpu", "single", L=chain.L, m=opts.m, prec=opts.prec, grad=opts.grad)
    return search(key, single_candidates(chain.L, opts.prec, sms or 152), timer, cache_path, force)


# ---------------------------------------------------------------- parity-excitation subspaces
def sector_candidates(D: int, prec: str, sms: int) -> list[dict]:
    """Threads per CTA that cover D (0: the library's choice) x grid (0: every CTA that fits)."""
    rows = {128: 4, 256: 10 if prec == "c64" else 8, 512: 8}
    shapes = [0] + [nt for nt, r in rows.items() if nt * r >= D]
    out = []
    for nt in shapes:
        for ctas in (0, sms):
            out.append(dict(block_threads=nt, ctas=ctas))
    return out


def tune_sector(spec: api.SectorSpec, opts: api.Options, B: int, u, psi0, target, device=None, repeats: int = 1,
                cache_path: str | None = None, force: bool = False, timer=None, gpu: str | None = None,
                sms: int | None = None) -> dict:
    """Fastest (block_threads, ctas) for B pulses in this subspace (milliseconds per launch)."""
    D = api.sector_dim(spec)
    if timer is None:
        dev, gpu, sms = _gpu(device)

        def timer(cand):
            s = dataclasses.replace(spec, block_threads=cand["block_threads"])
            eng = api.KGrapeSector(s, dataclasses.replace(opts, ctas=cand["ctas"]), B=B, device=dev)
            try:
                def run():
                    eng.evaluate(u, psi0, target)
                ms = _time_events(run, repeats, eng.stream)
                eng.sync()
                return ms
            finally:
                eng.close()
    key = cache_key(gpu or "gpu", "sector", D=D, B=B, m=opts.m, prec=opts.prec, grad=opts.grad)
    return search(key, sector_candidates(D, opts.prec, sms or 152), timer, cache_path, force)


# ---------------------------------------------------------------- batched evaluations
def signature(chains, opts: api.Options) -> str:
    h = hashlib.sha256()
    h.update(repr((opts.N, opts.m, opts.dt, opts.prec, opts.grad, opts.ckpt_every)).encode())
    for c in chains:
        h.update(repr((c.L, c.hc_kind, c.hc_site, c.hc_mask)).encode())
    return h.hexdigest()[:16]


def batch_candidates(sms: int) -> list[dict]:
    out = []
    for ctas in sorted({sms, (sms // 8) * 8, sms // 2}, reverse=True):
        for tpc in (2, 1):
            out.append(dict(ctas=ctas, tiles_per_cta=tpc))
    return out


def tune_batch(chains, opts: api.Options, u, psi0, target, device=None, repeats: int = 2,
               cache_path: str | None = None, force: bool = False, timer=None, gpu: str | None = None,
               sms: int | None = None) -> dict:
    """Fastest schedule {ctas, tiles_per_cta, ms} for this batch (cached by the batch's signature)."""
    if timer is None:
        dev, gpu, sms = _gpu(device)

        def timer(cand):
            b = api.KGrapeBatch(chains, opts, u, psi0, target, device=dev, **cand)
            try:
                ms = _time_events(b.launch, repeats, b.stream)
                b.sync()
                return ms
            finally:
                b.close()
    key = cache_key(gpu or "gpu", "batch", sig=signature(chains, opts))
    return search(key, batch_candidates(sms or 152), timer, cache_path, force)
