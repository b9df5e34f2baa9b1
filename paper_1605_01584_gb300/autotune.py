"""Tuner for the tensor-core kernels' knobs (pcc_set_tuning).

The knobs never change results, only speed:
  stage_k    K per shared-memory ring stage (32: 4 stages, 6 in the 2-SM
             pair form; 64: 2 stages, 3 in the pair form)
  pair_mma   1 = CTA pairs running one 2-SM MMA (each CTA loads half of
             the column operand), 0 = independent CTAs; the
             cluster knob follows it (2 with pairs, 1 without)
  band_rows  super-tile rows per band of the pair schedule
and the batched work split's cost model (cycles per unit c0, per K block and
product c1).

``tune_pairs(n, l)`` times every candidate on a synthetic matrix of that
shape with CUDA events and records the fastest in a JSON cache (one entry
per shape bucket: n rounded to a power of two, padded l, split form);
``apply(n, l, prec)`` loads the best known setting for the nearest bucket.
``calibrate_batched()`` fits c0, c1 from single-matrix timings at two row
lengths.  The cache lives at $PCC_TUNE_CACHE, else
~/.cache/paper_1605_01584_gb300/tune.json.
"""
from __future__ import annotations

import itertools
import json
import math
import numbers
import os
import statistics

from . import (PccError, load, pcc_allpairs_upper, pcc_get_tuning,
               pcc_set_tuning, pcc_standardize)

DEFAULT_CANDIDATES = {
    "stage_k": (32, 64),
    "pair_mma": (1, 0),
    "band_rows": (16, 32, 64),
}


def cache_path() -> str:
    p = os.environ.get("PCC_TUNE_CACHE")
    if p:
        return p
    return os.path.join(os.path.expanduser("~"), ".cache",
                        "paper_1605_01584_gb300", "tune.json")


def bucket(n: int, l: int, prec: str) -> str:
    """Shape bucket: n to the nearest power of two, l padded to 64."""
    nb = 1 << max(1, round(math.log2(max(n, 2))))
    lp = (l + 63) // 64 * 64
    return f"n{nb}_l{lp}_{prec}"


def load_cache(path: str | None = None) -> dict:
    path = path or cache_path()
    try:
        with open(path) as f:
            d = json.load(f)
        return d if isinstance(d, dict) else {}
    except (OSError, ValueError):
        return {}


def save_cache(cache: dict, path: str | None = None) -> None:
    path = path or cache_path()
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def _usable(entry) -> bool:
    """An entry written by tune_pairs: a 'best' record with every knob that
    apply() sets (a truncated or hand-edited cache is skipped, not fatal)."""
    if not isinstance(entry, dict) or not isinstance(entry.get("best"), dict):
        return False
    return all(isinstance(entry["best"].get(k), numbers.Integral)
               for k in ("stage_k", "cluster", "band_rows"))


def lookup(n: int, l: int, prec: str, cache: dict | None = None):
    """Best known knobs for (n, l, prec): the exact bucket, else the entry
    with the same split and padded l whose n is closest (log scale)."""
    cache = load_cache() if cache is None else cache
    key = bucket(n, l, prec)
    if _usable(cache.get(key)):
        return cache[key]["best"]
    lp = (l + 63) // 64 * 64
    best, dist = None, None
    for k, v in cache.items():
        if not k.endswith(f"_l{lp}_{prec}") or not _usable(v):
            continue
        nb = int(k.split("_")[0][1:])
        d = abs(math.log2(nb) - math.log2(max(n, 2)))
        if dist is None or d < dist:
            best, dist = v["best"], d
    return best


def lookup_batched(n: int, l: int, prec: str, cache: dict | None = None,
                   stage_k: int = 64):
    """(pair, band_rows) for one matrix of a batched launch: the fastest
    timed candidate with the batched kernel's stage size (stage_k, the
    current knob) in the entry lookup() would use; None without one."""
    cache = load_cache() if cache is None else cache
    key = bucket(n, l, prec)
    entry = cache.get(key) if _usable(cache.get(key)) else None
    if entry is None:
        lp = (l + 63) // 64 * 64
        dist = None
        for k, v in cache.items():
            if not k.endswith(f"_l{lp}_{prec}") or not _usable(v):
                continue
            d = abs(math.log2(int(k.split("_")[0][1:])) -
                    math.log2(max(n, 2)))
            if dist is None or d < dist:
                entry, dist = v, d
    if entry is None:
        return None
    runs = [r for r in entry.get("all", []) if isinstance(r, dict) and
            r.get("stage_k") == stage_k and
            isinstance(r.get("ms"), (int, float))]
    if not runs:
        return None
    b = min(runs, key=lambda r: r["ms"])
    return (1 if b.get("pair_mma") else 0, int(b["band_rows"]))


def tune_batched(shapes, prec: str = "auto", reps: int = 3,
                 bands=(8, 16, 32), path: str | None = None) -> dict:
    """Tune every distinct shape bucket of a batch (the current stage size,
    CTA pairs or single CTAs, the given band heights) on a synthetic matrix
    of the first shape of that bucket, and cache the results; returns
    bucket -> entry."""
    sk = pcc_get_tuning()["stage_k"]
    done = {}
    for n, l in shapes:
        key = bucket(n, l, "?")[:-2]
        if key in done:
            continue
        done[key] = tune_pairs(n, l, prec, reps=reps, path=path,
                               candidates={"stage_k": (sk,),
                                           "pair_mma": (1, 0),
                                           "band_rows": tuple(bands)})
    return done


def apply(n: int, l: int, prec: str, cache: dict | None = None) -> bool:
    """Set the library's knobs to the best known values for this shape;
    False (nothing changed) if the cache has no entry for it."""
    b = lookup(n, l, prec, cache)
    if not b:
        return False
    pcc_set_tuning(stage_k=b["stage_k"], cluster=b["cluster"],
                   band_rows=b["band_rows"], pair_mma=b.get("pair_mma"))
    return True


def _time_ms(fn, reps: int) -> float:
    import torch
    fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    return statistics.median(ts)


def tune_pairs(n: int, l: int, prec: str = "auto", candidates=None,
               reps: int = 5, seed: int = 0, save: bool = True,
               path: str | None = None) -> dict:
    """Time every knob combination on an n x l matrix and cache the best."""
    import torch
    load()
    cand = dict(DEFAULT_CANDIDATES)
    cand.update(candidates or {})
    g = torch.Generator(device="cuda").manual_seed(seed)
    X = torch.rand((n, l), device="cuda", generator=g)
    Z = pcc_standardize(X, prec)
    resolved = {2: "bf16x3", 3: "fp16x3s", 4: "bf16x4", 5: "bf16x1"}.get(
        Z.info()["prec"], str(prec))
    R = torch.empty(n * (n - 1) // 2, device="cuda")
    before = pcc_get_tuning()
    results = []
    try:
        for sk, pm, bd in itertools.product(
                cand["stage_k"], cand["pair_mma"], cand["band_rows"]):
            cl = 2 if pm else 1
            pcc_set_tuning(stage_k=sk, cluster=cl, band_rows=bd, pair_mma=pm)
            ms = _time_ms(lambda: pcc_allpairs_upper(Z, R), reps)
            results.append({"stage_k": sk, "cluster": cl, "pair_mma": pm,
                            "band_rows": bd, "ms": ms})
    finally:
        pcc_set_tuning(before["stage_k"], before["cluster"],
                       before["band_rows"], pair_mma=before["pair_mma"])
    best = min(results, key=lambda r: r["ms"])
    entry = {"n": n, "l": l, "prec": resolved, "best": best,
             "all": results}
    if save:
        cache = load_cache(path)
        cache[bucket(n, l, resolved)] = entry
        save_cache(cache, path)
    return entry


def calibrate_batched(n: int = 8192, ls=(64, 1024), reps: int = 5,
                      clock_ghz: float | None = None,
                      apply_now: bool = True) -> dict:
    """Fit the batched work split's cost model t_unit = c0 + c1 * kblocks *
    products (in cycles) from single-matrix timings at two row lengths."""
    import torch
    load()
    if clock_ghz is None:
        clock_ghz = 1.9  # only the ratio c0 : c1 matters to the work split
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    pts = []
    for l in ls:
        X = torch.rand((n, l), device="cuda")
        Z = pcc_standardize(X, "bf16x3")
        R = torch.empty(n * (n - 1) // 2, device="cuda")
        ms = _time_ms(lambda: pcc_allpairs_upper(Z, R), reps)
        m = -(-n // 256)
        units = m * (m + 1)
        per_unit_cycles = ms * 1e-3 * clock_ghz * 1e9 * sms / units
        kblocks = Z.info()["lpad"] // 32
        pts.append((kblocks * 3, per_unit_cycles))
    (x0, y0), (x1, y1) = pts
    c1 = max((y1 - y0) / max(x1 - x0, 1), 1.0)
    c0 = max(y0 - c1 * x0, 1.0)
    if apply_now:
        pcc_set_tuning(cost_c0=c0, cost_c1=c1)
    return {"c0": c0, "c1": c1, "points": pts, "clock_ghz": clock_ghz}
