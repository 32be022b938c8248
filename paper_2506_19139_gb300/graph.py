"""Batched training step captured in a CUDA graph (the batched path of the compositing core).

A RenderStep holds a fixed forward + backward render over any number of views: the scene
tensors, cameras, upstream gradients and parameter-gradient buffers are held by reference, so a
graph captured once replays on whatever values those tensors hold. The library renders all views of
one call with one preprocess, one binning pass, one tile sort and one composite launch over the
(view, tile) pairs of all views; the graph removes the remaining host work. The captured forward
runs with SOF_FLAG_ASYNC (no host round trip), sized by an eager synchronous run first. Its
capacities then stay fixed, so each replay must be checked with dropped() (or ok()) before its
results are used.
"""
from __future__ import annotations

import dataclasses

import torch

from . import _lib as L
from .render import (RenderOptions, Workspace, _out_c, _stream, alloc_outputs, cameras_to_c, render_forward_raw,
                     scene_to_c)

GRAD_KEYS = ("color", "depth", "exact_depth", "median_depth", "normal", "opacity")


class RenderStep:
    def __init__(self, scene_tensors, cams, opts: RenderOptions | None = None, grad_in: dict | None = None,
                 ws: Workspace | None = None):
        self.ts = list(scene_tensors)
        dev = self.ts[0].device
        self.cams = list(cams)
        self.opts = opts or RenderOptions()
        self.scene_c = scene_to_c(*self.ts)
        self.cams_c = cameras_to_c(self.cams)
        self.opts_sync = dataclasses.replace(self.opts, async_mode=False).to_c()
        self.opts_async = dataclasses.replace(self.opts, async_mode=True).to_c()
        self.outs = alloc_outputs(self.cams, dev, self.opts.median_depth)
        self.grads = [torch.zeros_like(t) for t in self.ts]
        self.grad_in = dict(grad_in or {})
        self.gin = L.sof_render_grad_in()
        for k in GRAD_KEYS:
            t = self.grad_in.get(k)
            setattr(self.gin, "d_median_depth" if k == "median_depth" else
                    ("d_exact_depth" if k == "exact_depth" else f"d_{k}"), 0 if t is None else t.data_ptr())
        self.sg = L.sof_scene_grad()
        g = self.grads
        self.sg.d_means, self.sg.d_log_scales, self.sg.d_quats = g[0].data_ptr(), g[1].data_ptr(), g[2].data_ptr()
        self.sg.d_opacity_logits, self.sg.d_sh = g[3].data_ptr(), g[4].data_ptr()
        self.ws = ws or Workspace(dev)
        self.graph = None

    def _bwd(self, opts_c):
        L.check(L.sof_render_bwd(self.scene_c, self.cams_c, len(self.cams), opts_c, _out_c(self.outs), self.gin,
                                 self.sg, self.ws.handle, _stream()), "sof_render_bwd", self.ws.handle)

    def run(self):
        """Eager step: synchronous forward (grows the workspace as needed), then the backward."""
        for t in self.grads:
            t.zero_()
        render_forward_raw(self.scene_c, self.cams_c, len(self.cams), self.opts_sync, self.outs, self.ws)
        self._bwd(self.opts_sync)

    def _run_async(self):
        for t in self.grads:
            t.zero_()
        L.check(L.sof_render_fwd(self.scene_c, self.cams_c, len(self.cams), self.opts_async, _out_c(self.outs),
                                 self.ws.handle, _stream()), "sof_render_fwd", self.ws.handle)
        self._bwd(self.opts_async)

    def capture(self):
        """Size everything with an eager run, then capture the asynchronous step in a CUDA graph."""
        self.run()
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self._run_async()
        self.graph = g
        return self

    def replay(self):
        if self.graph is None:
            raise RuntimeError("capture() first")
        self.graph.replay()

    def stats(self) -> dict:
        torch.cuda.synchronize()  # a replay runs on the current stream, not the capture stream
        return self.ws.stats()

    def dropped(self) -> int:
        """Pairs or visible records the last step could not hold (its results are invalid if > 0)."""
        return int(self.stats()["n_dropped"])

    def ok(self) -> bool:
        return self.dropped() == 0
