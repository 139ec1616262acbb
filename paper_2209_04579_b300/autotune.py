"""Autotuner for the tunable launch parameters.

It times each candidate with CUDA events on the current stream (after a
warm-up call) and checks that every candidate produces identical bytes. The
fastest candidate is cached in a JSON file keyed by GPU name, operator and
size class (log2 of the row count). The cache lives at
$TQP_AUTOTUNE_CACHE, else ~/.cache/tqp/autotune.json.

Tuned parameters:
  batched  -- fact rows per thread of the batched probe tile (4, 8, 16);
  learned  -- number of learned buckets B (about n/512 .. n/4096, powers of two),
              for the learned group-by and, through the same search with its
              own candidates, for the star join's learned dimension sorts;
  sort     -- rows per thread of the radix sort's tiles, per key width
              (8, 12, 16 for 32-bit keys; 6, 8, 12 for 64-bit keys), set
              process-wide with tqp_sort_tiles.
The radix digit is 8 bits by construction (one thread per digit value in
each pass), so the digit width is not a tuned parameter.
"""
from __future__ import annotations

import json
import math
import os

import torch

from . import tqp

_CACHE_PATH = os.environ.get("TQP_AUTOTUNE_CACHE",
                             os.path.join(os.path.expanduser("~"), ".cache", "tqp", "autotune.json"))


def _load():
    try:
        with open(_CACHE_PATH) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(d):
    try:
        os.makedirs(os.path.dirname(_CACHE_PATH), exist_ok=True)
        with open(_CACHE_PATH, "w") as f:
            json.dump(d, f, indent=1, sort_keys=True)
    except OSError:
        pass


def _key(op: str, rows: int) -> str:
    return f"{torch.cuda.get_device_name()}|{op}|{int(math.log2(max(rows, 1)))}"


def _time(fn, reps=3):
    fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    best = float("inf")
    for _ in range(reps):
        e0.record()
        fn()
        e1.record()
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return best


def _flat(o):
    for t in o:
        if isinstance(t, (list, tuple)):
            yield from _flat(t)
        else:
            yield t


def _fingerprint(outs):
    return [tuple(t.cpu().numpy().tobytes() for t in _flat(o)) for o in outs]


def tune_batched(problems, shape, cap=64, candidates=(4, 8, 16), force=False):
    """Best probe_items for one batched call; results of all candidates must agree."""
    rows = sum(int(p[0][0].numel()) for p in problems)
    cache = _load()
    k = _key("batched", rows)
    if not force and k in cache:
        return int(cache[k]["best"]), cache[k]
    times, ref = {}, None
    for c in candidates:
        times[c] = _time(lambda c=c: tqp.tqp_star_agg_batched(shape, problems, cap=cap, probe_items=c))
        fp = _fingerprint(tqp.tqp_star_agg_batched(shape, problems, cap=cap, probe_items=c))
        if ref is None:
            ref = fp
        elif fp != ref:
            raise RuntimeError(f"batched results differ between tile choices ({c})")
    best = min(times, key=times.get)
    cache[k] = {"best": best, "ms": {str(c): t for c, t in times.items()}}
    _store(cache)
    return best, cache[k]


def tune_learned(run, rows, candidates=None, force=False, op="learned"):
    """Best bucket count for the learned group-by (op names the call for
    the cache).  run(B) performs one call and returns its outputs (for the
    identity check)."""
    cache = _load()
    k = _key(op, rows)
    if not force and k in cache:
        return int(cache[k]["best"]), cache[k]
    if candidates is None:
        # from about 512 rows per bucket (most buckets sorted by one warp)
        # down to about 4096 (buckets sorted by one block; the steps of the
        # bucket function fit in shared memory up to 2^15 buckets)
        base = 256
        while base < (1 << 17) and base * 512 < rows:
            base <<= 1
        candidates = sorted({max(256, base >> s) for s in range(4)})
    times, ref = {}, None
    for b in candidates:
        times[b] = _time(lambda b=b: run(b))
        fp = _fingerprint([run(b)[:3]])
        if ref is None:
            ref = fp
        elif fp != ref:
            raise RuntimeError(f"learned results differ between bucket counts ({b})")
    best = min(times, key=times.get)
    cache[k] = {"best": best, "ms": {str(b): t for b, t in times.items()}}
    _store(cache)
    return best, cache[k]


def tune_sort(keys, vals=None, force=False):
    """Best sort tile for keys of this width (a representative input of the
    sorts to come), set with tqp_sort_tiles; every candidate must sort
    identically."""
    wide = keys.element_size() > 4
    cands = (6, 8, 12) if wide else (8, 12, 16)
    cache = _load()
    k = _key("sort64" if wide else "sort32", keys.numel())
    if not force and k in cache:
        best = int(cache[k]["best"])
    else:
        times, ref = {}, None
        for c in cands:
            tqp.tqp_sort_tiles(0, c) if wide else tqp.tqp_sort_tiles(c, 0)
            times[c] = _time(lambda: tqp.tqp_sort_pairs(keys, vals))
            fp = _fingerprint([tqp.tqp_sort_pairs(keys, vals)])
            if ref is None:
                ref = fp
            elif fp != ref:
                raise RuntimeError(f"sort results differ between tile choices ({c})")
        best = min(times, key=times.get)
        cache[k] = {"best": best, "ms": {str(c): t for c, t in times.items()}}
        _store(cache)
    tqp.tqp_sort_tiles(0, best) if wide else tqp.tqp_sort_tiles(best, 0)
    return best, cache[k]
