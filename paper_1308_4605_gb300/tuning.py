"""Autotuned multigrid schedules, cached on disk.

stk_autotune (C ABI) times every admissible schedule -- the level from which
the single-block coarse kernel takes over, the level from which smoothing
runs as two-colour kernels, and the threads per block of the per-colour
Gauss-Seidel kernels -- on the handle's own grid and applies the fastest.  `tune` wraps it with a JSON cache keyed by device name, grid,
boundary conditions and precision, so each shape is timed once per machine.
Cache file: $STK_TUNING_CACHE, else ~/.cache/stokes_gb300/schedules.json.
"""
from __future__ import annotations

import json
import os

from . import stokes as S


def cache_path():
    p = os.environ.get("STK_TUNING_CACHE")
    if p:
        return p
    return os.path.join(os.path.expanduser("~"), ".cache", "stokes_gb300", "schedules.json")


def _key(solver, precision):
    import torch
    dev = torch.cuda.get_device_name(torch.cuda.current_device())
    stack = getattr(solver, "count", 1)
    return f"s4|{dev}|{solver.dim}|{'x'.join(map(str, solver.n[:solver.dim]))}|" \
           f"{','.join(map(str, solver.bc[:2 * solver.dim]))}|{precision}" + \
           (f"|stack{stack}" if stack > 1 else "")


def _load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def tune(solver, precision, path=None):
    """Apply the cached schedule for this shape, or autotune and cache it.
    The solver's coefficients must be set.  Returns the schedule."""
    path = path or cache_path()
    cache = _load(path)
    key = _key(solver, precision)
    if key in cache:
        sc = cache[key]
        S.stk_set_schedule(solver.handle, precision, sc["coarse_level"], sc["threads"],
                           sc["pair_level"], sc.get("grid_level"), sc.get("cluster_level"))
        return sc
    sc = S.stk_autotune(solver.handle, precision)
    cache = _load(path)
    cache[key] = sc
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + f".{os.getpid()}.tmp"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1, sort_keys=True)
        os.replace(tmp, path)
    except OSError:
        pass
    return sc
