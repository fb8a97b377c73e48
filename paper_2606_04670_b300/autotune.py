"""Autotuner for the launch shapes of lip_eval and lip_batch_eval.

The results of both calls do not depend on their launch shape (the tests check bitwise
equality), so the shape is chosen purely by measured time: every candidate is timed
with CUDA events on the launching stream, taking the median of several runs after a
warm-up, and the fastest is kept.

* ``tune_eval(model, Q)`` sweeps the scan kernel variant (queries per thread), the
  shared-memory tile (tile_groups) and the number of data splits of one data set,
  applies the best with ``lip_set_tuning`` and returns it.
* ``tune_batch(sets)`` sweeps the batch options (default tile, work items per resident
  block, persistent-grid waves) and returns the best ``lip_batch_options`` as a dict.

Results are cached in a JSON file keyed by the problem's shape and size buckets
(norm, constrained and free coordinates, log2 of N and of the query count), so a later
run reuses them without timing.
"""
from __future__ import annotations

import json
import math
import os
import statistics
from typing import Dict, Iterable, Optional

import numpy as np

DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuning", "b300_cache.json")


def _bucket(n: int) -> int:
    return int(math.floor(math.log2(max(1, n))))


PRUNED_DMAX = 8        # the pruned scan's instantiations (FP32, d <= 8, and unconstrained
PRUNED_UMAX = 16       # shapes up to d = 16)


def pruned_capable(model) -> bool:
    """FP32 handles whose shape has a pruned instantiation: d <= 8, or unconstrained up to 16."""
    from .lipfit import LIP_FP32
    c = 0 if model.mon is None else int((np.asarray(model.mon) != 0).sum())
    return model.precision == LIP_FP32 and (model.d <= PRUNED_DMAX or (c == 0 and model.d <= PRUNED_UMAX))


def eval_key(model, nq: int) -> str:
    c = 0 if model.mon is None else int((model.mon != 0).sum())
    # "eval6": shapes with the pruned scan (variants 6, 7: 16-point chunks skipped per
    # 32-query row, Hilbert order, nearest first) among their eight variants; "eval2":
    # the others (six FP32 variants, the FMA-pipe square roots)
    tag = "eval6" if pruned_capable(model) else "eval2"
    return f"{tag}/norm{model.norm}/C{c}/U{model.d - c}/prec{model.precision}/N2^{_bucket(model.N)}/Q2^{_bucket(nq)}"


def load_cache(path: Optional[str] = None) -> Dict:
    path = path or DEFAULT_CACHE
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def save_cache(cache: Dict, path: Optional[str] = None):
    path = path or DEFAULT_CACHE
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def _time(fn, reps: int = 3, warm: int = 1) -> float:
    import torch
    for _ in range(warm):
        fn()
    ts = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record()
        fn()
        b.record()
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    return statistics.median(ts)


def tune_eval(model, Q, tiles: Iterable[int] = (8, 16, 32, 64), splits: Iterable[int] = (0, 1, 2, 3, 4, 6, 8, 12, 16),
              variants: Optional[Iterable[int]] = None, cache: Optional[Dict] = None, reps: int = 3) -> Dict:
    """Time lip_eval on `model` for every (variant, tile_groups, splits); apply the fastest.
    The variants default to the eight of FP32 handles (queries per thread x the share of
    square roots on the FMA pipe, and the pruned scan, which ignores splits), to 0, 1 for
    FP64 handles and to 0-5 for tensor-core handles (epilogue warps x the launch form),
    which ignore tiles and splits."""
    from .lipfit import LIP_FP32, LIP_FP64
    tc = model.precision not in (LIP_FP32, LIP_FP64)
    if variants is None:
        variants = ((range(8) if pruned_capable(model) else range(6)) if model.precision == LIP_FP32
                    else (range(6) if tc else (0, 1)))
    if tc:
        tiles, splits = (32,), (0,)
    key = eval_key(model, Q.shape[0])
    if cache is not None and key in cache:
        best = cache[key]
        model.set_tuning(best["tile_groups"], best["splits"], best.get("variant", 0))
        return dict(best, cached=True)
    results = []
    for v in variants:
        for tg in tiles:
            for sp in (splits if v < 6 or tc else list(splits)[:1]):
                model.set_tuning(tg, sp, v)
                ms = _time(lambda: model.eval(Q, need=("g", "idx_up", "idx_lo")), reps=reps)
                results.append({"variant": model.tuning()["variant"], "tile_groups": tg, "splits": sp, "ms": ms,
                                "splits_used": model.tuning()["last_splits"]})
    best = min(results, key=lambda r: r["ms"])
    model.set_tuning(best["tile_groups"], best["splits"], best["variant"])
    rec = {"variant": best["variant"], "tile_groups": best["tile_groups"], "splits": best["splits"], "ms": best["ms"],
           "default_ms": next((r["ms"] for r in results
                               if r["tile_groups"] == 32 and r["splits"] == 0 and r["variant"] == 0), None),
           "candidates": len(results)}
    if cache is not None:
        cache[key] = rec
    return dict(rec, cached=False)


def batch_key(sets) -> str:
    n = len(sets)
    pairs = sum(int(s["Q"].shape[0]) * int(s["X"].shape[0]) for s in sets)
    return f"batch/sets{n}/pairs2^{_bucket(pairs)}"


def tune_batch(sets, tiles: Iterable[int] = (16, 32, 64), items: Iterable[int] = (2, 4, 8, 16),
               waves: Iterable[int] = (1,), cache: Optional[Dict] = None, reps: int = 2, outputs=None) -> Dict:
    """Time lip_batch_eval for every option combination; return the fastest options."""
    from .lipfit import LipBatch
    key = batch_key(sets)
    if cache is not None and key in cache:
        return dict(cache[key], cached=True)
    results = []
    for tg in tiles:
        for it in items:
            for wv in waves:
                b = LipBatch(sets, tile_groups=tg, items_per_block=it, waves=wv, outputs=outputs)
                ms = _time(b.eval, reps=reps)
                results.append({"tile_groups": tg, "items_per_block": it, "waves": wv, "ms": ms})
                b.close()
    best = min(results, key=lambda r: r["ms"])
    rec = {k: best[k] for k in ("tile_groups", "items_per_block", "waves", "ms")}
    rec["candidates"] = len(results)
    rec["default_ms"] = next((r["ms"] for r in results if r["tile_groups"] == 32 and r["items_per_block"] == 8
                              and r["waves"] == 1), None)
    if cache is not None:
        cache[key] = rec
    return dict(rec, cached=False)
