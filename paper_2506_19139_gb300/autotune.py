"""Autotuner for the composite's launch parameters: a thin front end of sof_autotune.

The composite kernel is instantiated for the screen tile edge (tile: 8, 16 or 32 pixels), the
records staged per shared-memory chunk (chunk) and the per-pixel pending-hit buffer size
(reorder_k); the best triple depends on the scene's depth complexity, the Gaussians' screen sizes
and the views' sizes. sof_autotune times a full forward + backward step for every instantiated
triple on the caller's own workload, with CUDA events on the current stream, and returns the
fastest. This module allocates the step's buffers, grows the workspace as the library asks, and
keeps the results per workload signature in memory; the library keeps them in a text file if a
path is given. Every candidate renders the same exact result: the parameters change only speed.
"""
from __future__ import annotations

import dataclasses

import torch

from . import _lib as L
from .render import RenderOptions, Workspace, _out_c, _stream, alloc_outputs, cameras_to_c, scene_to_c


def candidates():
    """The (tile, chunk, reorder_k) triples the library instantiates, in sof_autotune's order."""
    return tuple(L.sof_autotune_candidate(i) for i in range(L.SOF_AUTOTUNE_CANDIDATES))


_cache: dict = {}


def signature(scene_tensors, cams, views_per_call=None) -> str:
    means, sh = scene_tensors[0], scene_tensors[4]
    views = ",".join(f"{c.width}x{c.height}" for c in cams)
    return f"n={means.shape[0]};sh={sh.shape[1]};vpc={views_per_call or 0};views={views}"


def tune(scene_tensors, cams, base: RenderOptions | None = None, reps: int = 2, cache_path: str | None = None,
         views_per_call: int | None = None, ws: Workspace | None = None, max_retries: int = 4):
    """Fastest (tile, chunk, reorder_k) for this workload; returns (RenderOptions,
    {(tile, chunk, k): ms, or None where the library refuses the triple for this workload})."""
    base = base or RenderOptions()
    key = signature(scene_tensors, cams, views_per_call) + repr(dataclasses.astuple(base))
    if key in _cache:
        return _cache[key]
    dev = scene_tensors[0].device
    ts = list(scene_tensors)
    scene_c = scene_to_c(*ts)
    cams_c = cameras_to_c(cams)
    npx = sum(c.width * c.height for c in cams)
    outs = alloc_outputs(cams, dev, base.median_depth)
    d_color = torch.full((3 * npx,), 1e-3, device=dev)
    gin = L.sof_render_grad_in()
    gin.d_color = d_color.data_ptr()
    grads = [torch.zeros_like(t) for t in ts]
    sg = L.sof_scene_grad()
    sg.d_means, sg.d_log_scales, sg.d_quats = grads[0].data_ptr(), grads[1].data_ptr(), grads[2].data_ptr()
    sg.d_opacity_logits, sg.d_sh = grads[3].data_ptr(), grads[4].data_ptr()
    ws = ws or Workspace(dev)
    opts_c = dataclasses.replace(base, async_mode=True).to_c()
    if ws.buffer is None:
        ws.ensure(L.sof_render_workspace_size(scene_c, cams_c, min(len(cams), views_per_call or len(cams)), opts_c,
                                              1 << 16))
    for _ in range(max_retries):
        rc, best, ms = L.sof_autotune(scene_c, cams_c, len(cams), views_per_call or 0, opts_c, _out_c(outs), gin, sg,
                                      reps, cache_path, ws.handle, _stream())
        if rc == L.SOF_ERR_WORKSPACE_TOO_SMALL:
            ws.ensure(L.sof_workspace_required(ws.handle))
            continue
        L.check(rc, "sof_autotune", ws.handle)
        times = {c: (m if m >= 0 else None) for c, m in zip(candidates(), ms)}
        res = (dataclasses.replace(base, tile=best.tile, chunk=best.chunk, reorder_k=best.reorder_k), times)
        _cache[key] = res
        return res
    raise L.SOFError(L.SOF_ERR_WORKSPACE_TOO_SMALL, "sof_autotune")
