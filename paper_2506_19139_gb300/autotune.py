"""Autotuner for the composite's launch parameters.

The composite kernel is instantiated for the screen tile edge (tile: 8, 16 or 32 pixels), the
records staged per shared-memory chunk (chunk) and the per-pixel pending-hit buffer size
(reorder_k); the best triple depends on the scene's depth complexity, the Gaussians' screen sizes
and the views' sizes. tune() times a full forward + backward step for every instantiated triple on
the caller's own workload, with CUDA events on the current stream, and returns the fastest
RenderOptions. Results are cached per workload signature (Gaussian count, SH degree and view sizes)
in memory and, if a path is given, in a JSON file. Every candidate renders the same exact result:
the parameters change only speed.
"""
from __future__ import annotations

import dataclasses
import json
import os

import torch

from . import _lib as L
from .render import RenderOptions

# (tile, chunk, reorder_k) triples the library instantiates
CANDIDATES = ((16, 64, 16), (16, 32, 16), (16, 128, 16), (16, 64, 8), (16, 64, 32), (16, 32, 8), (16, 32, 32),
              (8, 64, 16), (8, 64, 32), (32, 64, 8), (32, 64, 16))

_cache: dict = {}


def signature(scene_tensors, cams) -> str:
    means, sh = scene_tensors[0], scene_tensors[4]
    views = ",".join(f"{c.width}x{c.height}" for c in cams)
    return f"n={means.shape[0]};sh={sh.shape[1]};views={views}"


def tune(scene_tensors, cams, base: RenderOptions | None = None, reps: int = 2, cache_path: str | None = None,
         candidates=CANDIDATES, views_per_call: int | None = None):
    """Fastest (tile, chunk, reorder_k) for this workload; returns (RenderOptions,
    {(tile, chunk, k): ms, or None where the library refuses the triple for this workload})."""
    from .graph import RenderStep
    base = base or RenderOptions()
    key = signature(scene_tensors, cams)
    if key not in _cache and cache_path and os.path.exists(cache_path):
        with open(cache_path) as f:
            _cache.update(json.load(f))
    if key in _cache:
        tl, ch, k = _cache[key]["best"]
        return dataclasses.replace(base, tile=tl, chunk=ch, reorder_k=k), {tuple(map(int, a.split(":"))): v
                                                                           for a, v in _cache[key]["ms"].items()}
    grad_in = {"color": torch.full((3 * sum(c.width * c.height for c in cams),), 1e-3,
                                   device=scene_tensors[0].device)}
    ws = None
    times = {}
    for tl, ch, k in candidates:
        step = RenderStep(scene_tensors, cams, dataclasses.replace(base, tile=tl, chunk=ch, reorder_k=k), grad_in,
                          ws, views_per_call)
        ws = step.ws  # one workspace for all candidates
        try:
            step.run()  # warm-up (sizes the workspace)
        except L.SOFError as e:
            if e.code != L.SOF_ERR_INVALID_ARG:
                raise
            # not usable for this workload (e.g. small tiles give more pairs than one call indexes)
            times[(tl, ch, k)] = None
            continue
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            step.run()
        e1.record()
        torch.cuda.synchronize()
        times[(tl, ch, k)] = e0.elapsed_time(e1) / reps
    usable = {t: v for t, v in times.items() if v is not None}
    if not usable:
        raise RuntimeError("no instantiated (tile, chunk, reorder_k) renders this workload")
    best = min(usable, key=usable.get)
    _cache[key] = {"best": list(best), "ms": {":".join(map(str, t)): v for t, v in times.items()}}
    if cache_path:
        with open(cache_path, "w") as f:
            json.dump(_cache, f, indent=1)
    return dataclasses.replace(base, tile=best[0], chunk=best[1], reorder_k=best[2]), times
