"""Launch-shape autotuner for ensembles (and single grids).

Times each candidate (steps per launch K, warps per block, rows per chunk,
steps per graph replay) on the live ensemble with CUDA events, keeps the
fastest, and caches the choice in a JSON file keyed by the device name and the
scenario shapes (``$FLOOD_AUTOTUNE_CACHE`` or
``~/.cache/paper_2204_10323_gb300/autotune.json``).  K = 0 is the single-step
stream kernel (warps and rows shape its blocks); K >= 1 the temporal-blocking
kernel with K steps per launch (rows per (chunk, strip) item of a 2^20-cell
grid, scaled by the square root of each grid's cells).  Every
candidate computes bit-identical depths and discharges, so tuning on the live
run does not change its trajectory; it only advances it.
"""
from __future__ import annotations

import json
import os
from typing import Iterable, Optional, Sequence, Tuple

import torch

Shape = Tuple[int, int, int, int]       # (K, warps, rows, steps per graph)


def cache_path() -> str:
    return os.environ.get("FLOOD_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "paper_2204_10323_gb300",
                                       "autotune.json"))


def _load(path: str) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _save(path: str, data: dict) -> None:
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)
        os.replace(tmp, path)
    except OSError:
        pass


def ensemble_key(ens) -> str:
    shapes = ",".join(f"{p.nx}x{p.ny}" for p in ens.problems)
    return f"v4|{torch.cuda.get_device_name()}|E{ens.problems[0].opts.epoch_steps}|{shapes}"


def default_candidates(E: int) -> Sequence[Shape]:
    stream = [(0, w, r, g) for w in (2, 4) for r in (32, 64, 128) for g in (E, 4 * E)]
    tiled = [(k, 2, r, g) for k in (2, 4) if E % k == 0 for r in (96, 128, 192, 256, 320) for g in (E, 4 * E)]
    return stream + tiled


def apply(ens, shape: Shape) -> None:
    k, w, r, g = shape
    ens.set_launch(w, r, g)
    if k > 0:
        ens.set_kernel(_kernels().KERNEL_TILED, k)
    else:
        ens.set_kernel(_kernels().KERNEL_STREAM, 0)


def _kernels():
    import paper_2204_10323_gb300 as F
    return F


def tune_ensemble(ens, candidates: Optional[Iterable[Shape]] = None, trial_steps: Optional[int] = None,
                  use_cache: bool = True) -> dict:
    """Pick and set the fastest launch shape; returns {shape, ms_per_step, trials}."""
    E = ens.problems[0].opts.epoch_steps
    key = ensemble_key(ens)
    path = cache_path()
    cache = _load(path) if use_cache else {}
    if use_cache and key in cache:
        apply(ens, tuple(cache[key]["shape"]))
        return dict(cache[key], cached=True)
    cands = list(candidates or default_candidates(E))
    # the ensemble's work runs on its own stream: the events must be recorded there
    stream = getattr(ens, "stream", None) or torch.cuda.current_stream()
    trials = []
    for shape in cands:
        apply(ens, shape)
        g = shape[3]
        steps = trial_steps or 2 * g
        steps = max(g, (steps // g) * g)
        ens.step(g)                        # capture + warm
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        ens.step(steps)
        b.record(stream)
        torch.cuda.synchronize()
        trials.append((tuple(shape), a.elapsed_time(b) / steps))
    best, ms = min(trials, key=lambda t: t[1])
    apply(ens, best)
    result = {"shape": list(best), "ms_per_step": ms, "trials": [[list(s), t] for s, t in trials]}
    if use_cache:
        cache[key] = result
        _save(path, cache)
    return dict(result, cached=False)
