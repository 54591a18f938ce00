"""The schedule autotuner's search and cache, with a fake timer (no GPU): it keeps the fastest
candidate, skips the ones the library refuses, keys the cache by (GPU, kind, size, m, precision,
gradient mode) and re-times only when asked."""
import json

import pytest

from paper_2010_03598_gb300 import api as A
from paper_2010_03598_gb300 import tune


def fake_timer(calls, refuse=()):
    def timer(cand):
        calls.append(dict(cand))
        if cand.get("tile_bits") in refuse:
            raise RuntimeError("refused")
        # fastest: tile_bits 12 on 128 CTAs
        return 1.0 + abs(cand.get("tile_bits", 0) - 12) + abs(cand.get("ctas", 0) - 128) / 100.0
    return timer


def test_single_search_picks_the_fastest_and_caches_it(tmp_path):
    path = str(tmp_path / "cache.json")
    chain, opts = A.ChainSpec(20), A.Options(400, 0.05, 20, prec="c64")
    calls = []
    best = tune.tune_single(chain, opts, None, None, None, cache_path=path, timer=fake_timer(calls),
                            gpu="GB300", sms=152)
    assert (best["tile_bits"], best["ctas"]) == (12, 128)
    assert len(calls) == len(tune.single_candidates(20, "c64", 152)) == len(best["trials"])
    assert {"tile_bits": 0, "ctas": 0} in [{k: t[k] for k in ("tile_bits", "ctas")} for t in best["trials"]]
    cache = json.load(open(path))
    key = tune.cache_key("GB300", "single", L=20, m=20, prec="c64", grad="centered")
    assert key in cache and cache[key]["tile_bits"] == 12
    # another pulse length of the same chain and options: served from the cache
    calls2 = []
    again = tune.tune_single(chain, A.Options(64, 0.1, 20, prec="c64"), None, None, None, cache_path=path,
                             timer=fake_timer(calls2), gpu="GB300", sms=152)
    assert calls2 == [] and again["tile_bits"] == 12
    # another m, precision, gradient mode or GPU: a new search
    for o, gpu in ((A.Options(400, 0.05, 16, prec="c64"), "GB300"), (A.Options(400, 0.05, 20, prec="c128"), "GB300"),
                   (A.Options(400, 0.05, 20, prec="c64", grad="zeroth"), "GB300"), (opts, "other")):
        calls3 = []
        tune.tune_single(chain, o, None, None, None, cache_path=path, timer=fake_timer(calls3), gpu=gpu, sms=152)
        assert calls3
    # force: timed again
    calls4 = []
    tune.tune_single(chain, opts, None, None, None, cache_path=path, timer=fake_timer(calls4), gpu="GB300", sms=152,
                     force=True)
    assert calls4


def test_refused_candidates_are_skipped(tmp_path):
    path = str(tmp_path / "cache.json")
    calls = []
    best = tune.tune_single(A.ChainSpec(20), A.Options(8, 0.05, 20), None, None, None, cache_path=path,
                            timer=fake_timer(calls, refuse=(12,)), gpu="g", sms=152)
    assert best["tile_bits"] != 12
    assert any(t["ms"] is None for t in best["trials"])
    with pytest.raises(RuntimeError):
        tune.search("k", [dict(a=1)], lambda c: (_ for _ in ()).throw(RuntimeError("no")), str(tmp_path / "c2.json"))


def test_candidate_lists():
    single = tune.single_candidates(20, "c64", 152)
    assert single[0] == dict(tile_bits=0, ctas=0)
    assert dict(tile_bits=12, ctas=128) in single and dict(tile_bits=11, ctas=152) in single
    assert all(c["tile_bits"] <= 11 for c in tune.single_candidates(20, "c128", 152))
    assert all(c["tile_bits"] <= 8 for c in tune.single_candidates(8, "c64", 152))
    sec = tune.sector_candidates(2445, "c64", 152)
    assert {c["block_threads"] for c in sec} == {0, 256, 512}  # 128 x 4 rows cannot cover D = 2445
    assert {c["block_threads"] for c in tune.sector_candidates(511, "c64", 152)} == {0, 128, 256, 512}
    assert {c["block_threads"] for c in tune.sector_candidates(2445, "c128", 152)} == {0, 512}
    # float-float vectors take the complex128 path's shapes (16-byte amplitudes)
    assert {c["block_threads"] for c in tune.sector_candidates(2445, "ff", 152)} == {0, 512}
    assert {c["block_threads"] for c in tune.sector_candidates(511, "ff", 152)} == {0, 128, 256, 512}
    bc = tune.batch_candidates(152)
    assert len(bc) == 4 and len(tune.batch_candidates(150)) == 6  # 152 SMs are already a multiple of 8
    assert all(c["ctas"] <= 152 for c in tune.single_candidates(20, "c64", 152))


def test_sector_search_uses_the_subspace_dimension(tmp_path):
    path = str(tmp_path / "cache.json")
    spec = A.SectorSpec(14, 4, 1)
    seen = []
    best = tune.tune_sector(spec, A.Options(64, 0.5, 10), 8, None, None, None, cache_path=path,
                            timer=lambda c: seen.append(c) or (2.0 if c["block_threads"] == 256 else 3.0), gpu="g",
                            sms=152)
    assert best["block_threads"] == 256
    key = tune.cache_key("g", "sector", D=A.sector_dim(spec), B=8, m=10, prec="c64", grad="centered")
    assert key in json.load(open(path))
