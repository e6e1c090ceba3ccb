"""Autotuner for the solve schedule.

For a single-system plan it times every candidate (mode, rows per warp, rhs
tile) with CUDA events and keeps the fastest (winners are cached in a JSON
file keyed by size class: ``SPTRSV_TUNE_CACHE`` or
``~/.cache/sptrsv_gb300/tune.json``).  For a batched plan, whose time is a
makespan, it first sets one right-hand-side tile for every system, then
refines rows per warp and tile per size class (bucketed average row length
and number of right-hand sides) by coordinate descent.
"""
from __future__ import annotations

import json
import math
import os

import numpy as np
import torch

from . import _lib as L
from .api import BatchPlan, Plan

CANDIDATE_MODES = ("level", "syncfree", "block", "hybrid")
CANDIDATE_RPW = (1, 4, 8, 16, 32)


def _cache_path():
    p = os.environ.get("SPTRSV_TUNE_CACHE")
    if p:
        return p
    return os.path.join(os.path.expanduser("~"), ".cache", "sptrsv_gb300", "tune.json")


def _load_cache():
    try:
        with open(_cache_path()) as f:
            return json.load(f)
    except Exception:
        return {}


def _store_cache(c):
    p = _cache_path()
    try:
        os.makedirs(os.path.dirname(p), exist_ok=True)
        with open(p + ".tmp", "w") as f:
            json.dump(c, f, indent=1, sort_keys=True)
        os.replace(p + ".tmp", p)
    except OSError:
        pass


def _bucket(v):
    return int(round(math.log2(max(v, 1e-9)))) if v > 0 else -99


def size_class(n, nnz, nlevels, k, dtype) -> str:
    """Size class of a system: log2 buckets of n, row length, level width, k."""
    width = n / max(nlevels, 1)
    return (f"{str(dtype).split('.')[-1]}:n{_bucket(n)}:r{_bucket(nnz / max(n, 1))}"
            f":w{_bucket(width)}:k{_bucket(k)}")


def time_call(fn, reps=5, warmup=2) -> float:
    """Median milliseconds of fn() on the current stream (CUDA events)."""
    for _ in range(warmup):
        fn()
    s = torch.cuda.current_stream()
    ts = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(s)
        fn()
        b.record(s)
        b.synchronize()
        ts.append(a.elapsed_time(b))
    return float(np.median(ts))


def tune_plan(plan: Plan, b: torch.Tensor, modes=CANDIDATE_MODES, rpws=CANDIDATE_RPW,
              kts=None, use_cache=True, reps=5):
    """Times every candidate on the right-hand side b and applies the best."""
    n, k = plan.A.n, (b.shape[1] if b.dim() == 2 else 1)
    info = plan.info()
    key = size_class(n, plan.A.nnz, info["nlevels"], k, plan.A.dtype)
    cache = _load_cache() if use_cache else {}
    if key in cache:
        c = cache[key]
        plan.set(c["mode"], c["rows_per_warp"], c["rhs_tile"])
        return dict(key=key, best=c, cached=True, table=[])
    if kts is None:
        kts = [t for t in (1, 2, 4, 8, 16) if t <= max(1, 1 << math.ceil(math.log2(k)))] or [1]
    x = torch.empty(n, k, dtype=b.dtype, device=b.device)
    b2 = b.view(n, k)
    table = []
    for mode in modes:
        for rpw in rpws:
            for kt in kts:
                plan.set(mode, rpw, kt)
                ms = time_call(lambda: plan.solve(b2, out=x), reps=reps)
                table.append(dict(mode=mode, rows_per_warp=rpw, rhs_tile=kt, ms=ms))
    best = min(table, key=lambda r: r["ms"])
    plan.set(best["mode"], best["rows_per_warp"], best["rhs_tile"])
    if use_cache:
        cache = _load_cache()
        cache[key] = best
        _store_cache(cache)
    return dict(key=key, best=best, cached=False, table=table)


def batch_classes(bplan: BatchPlan):
    """Size class label (average row length bucket, k bucket) of each system."""
    labels = []
    for A, k in zip(bplan.mats, bplan.nrhs):
        labels.append(f"r{_bucket(A.nnz / max(A.n, 1))}:k{_bucket(k)}")
    return labels


def tune_batch(bplan: BatchPlan, b: torch.Tensor, candidates=(8, 16, 32), tiles=(2, 4, 8), reps=3,
               rounds=1, direction="forward", schedules=("inorder", "level")):
    """Rows-per-warp, right-hand-side tile and schedule (in row order or
    level by level) of the batched solve in one direction ("forward": the
    solve; "transpose": the transpose solve of the adjoint, which has its
    own geometry and its own timing).  The batch time is a makespan, so the
    search first sets one tile width for every system, then refines per
    size class (coordinate descent: each class tries every candidate of one
    knob with everything else fixed).  A rows-per-warp of 0 keeps the plan's
    default for that system; the level schedule ignores it."""
    if direction not in ("forward", "transpose"):
        raise ValueError("direction must be 'forward' or 'transpose'")
    labels = batch_classes(bplan)
    classes = sorted(set(labels))
    x = torch.empty_like(b)
    log = []
    run = bplan.solve if direction == "forward" else bplan.solve_transpose

    def apply(choice):
        bplan.set_geometry([choice[l][0] for l in labels], [choice[l][1] for l in labels], direction=direction)
        bplan.set_schedule([choice[l][2] for l in labels], direction=direction)

    def measure(choice):
        try:
            apply(choice)
        except L.SpTRSVError:
            return None
        return time_call(lambda: run(b, out=x), reps=reps)

    best, best_ms = None, float("inf")
    for t in tiles:
        choice = {c: [0, t, "inorder"] for c in classes}
        ms = measure(choice)
        log.append(dict(step="uniform", rhs_tile=t, ms=ms))
        if ms is not None and ms < best_ms:
            best, best_ms = choice, ms
    if best is None:
        raise L.SpTRSVError(L.SPTRSV_ENOTSUP, "tune_batch: no candidate right-hand-side tile fits this batch")
    choice = best
    for _ in range(rounds):
        for c in classes:
            for knob, cands in ((0, candidates), (1, tiles), (2, schedules)):
                keep = choice[c][knob]
                for cand in cands:
                    if cand == keep:
                        continue
                    choice[c][knob] = cand
                    ms = measure(choice)
                    log.append(dict(cls=c, knob=("rows_per_warp", "rhs_tile", "schedule")[knob], value=cand, ms=ms))
                    if ms is not None and ms < best_ms * 0.995:
                        best_ms, keep = ms, cand
                choice[c][knob] = keep
    apply(choice)
    return dict(choice={c: dict(rows_per_warp=v[0], rhs_tile=v[1], schedule=v[2]) for c, v in choice.items()},
                ms=best_ms,
                log=log, direction=direction)
