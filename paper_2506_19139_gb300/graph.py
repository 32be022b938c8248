"""Batched training step, and the opacity query over all views, captured in CUDA graphs (the batched
path of the compositing core).

A RenderStep holds a fixed forward + backward render over any number of views. The scene
tensors, cameras, upstream gradients and parameter-gradient buffers are held by reference, so a
graph captured once replays on whatever values those tensors hold.

The library renders all views of one call with one preprocess, one binning pass, one tile sort
and one composite launch over the (view, tile) pairs of all views. Views are grouped into calls of
`views_per_call` (default: all views in one call): one call indexes its (Gaussian, tile) pairs with
32 bits, and its workspace grows with the views it holds. The groups run one after the other on
one workspace, and their gradients accumulate into the same buffers.

The graph removes the remaining host work: capture() hands the step to sof_graph_capture, which
sizes the workspace (sof_workspace_reserve per call), runs the step once and captures its
stream-ordered forwards and backwards (no host round trip) into a CUDA graph; replay() is
sof_graph_launch on the current stream. The capacities then stay fixed, so check each replay with
dropped() (or ok()) before using its results.
"""
from __future__ import annotations

import dataclasses

import torch

from . import _lib as L
from .render import RenderOptions, Workspace, _out_c, _stream, alloc_outputs, cameras_to_c, render_forward_raw, scene_to_c

_GIN_FIELDS = {"color": "d_color", "depth": "d_depth", "exact_depth": "d_exact_depth",
               "median_depth": "d_median_depth", "normal": "d_normal", "opacity": "d_opacity"}
_THREE = ("color", "normal")


class RenderStep:
    def __init__(self, scene_tensors, cams, opts: RenderOptions | None = None, grad_in: dict | None = None,
                 ws: Workspace | None = None, views_per_call: int | None = None):
        self.ts = list(scene_tensors)
        dev = self.ts[0].device
        self.cams = list(cams)
        self.opts = opts or RenderOptions()
        self.scene_c = scene_to_c(*self.ts)
        self.opts_sync = dataclasses.replace(self.opts, async_mode=False).to_c()
        self.opts_async = dataclasses.replace(self.opts, async_mode=True).to_c()
        self.outs = alloc_outputs(self.cams, dev, self.opts.median_depth)
        self.grads = [torch.zeros_like(t) for t in self.ts]
        self.grad_in = dict(grad_in or {})
        self.sg = L.sof_scene_grad()
        g = self.grads
        self.sg.d_means, self.sg.d_log_scales, self.sg.d_quats = g[0].data_ptr(), g[1].data_ptr(), g[2].data_ptr()
        self.sg.d_opacity_logits, self.sg.d_sh = g[3].data_ptr(), g[4].data_ptr()
        self.ws = ws or Workspace(dev)
        self.graph = None
        self.vpc = views_per_call or len(self.cams)
        self.cams_all_c = cameras_to_c(self.cams)
        self.outs_all_c = _out_c(self.outs)
        self.gin_all = L.sof_render_grad_in()
        for k, field in _GIN_FIELDS.items():
            t = self.grad_in.get(k)
            setattr(self.gin_all, field, 0 if t is None else t.data_ptr())
        # per call: its cameras, and its slices of the packed outputs and upstream gradients
        vpc = self.vpc
        self.calls = []
        p0 = 0
        for i in range(0, len(self.cams), vpc):
            cs = self.cams[i:i + vpc]
            p1 = p0 + sum(c.width * c.height for c in cs)

            def sl(t, k, a=p0, b=p1):
                if t is None:
                    return None
                return t[3 * a:3 * b] if k in _THREE else t[a:b]
            outs = {k: sl(v, k) for k, v in self.outs.items()}
            gin = L.sof_render_grad_in()
            keep = {}
            for k, field in _GIN_FIELDS.items():
                t = sl(self.grad_in.get(k), k)
                keep[k] = t
                setattr(gin, field, 0 if t is None else t.data_ptr())
            self.calls.append({"cams": cs, "cams_c": cameras_to_c(cs), "outs": outs, "outs_c": _out_c(outs),
                               "gin": gin, "keep": keep})
            p0 = p1

    def _bwd(self, call, opts_c):
        L.check(L.sof_render_bwd(self.scene_c, call["cams_c"], len(call["cams"]), opts_c, call["outs_c"], call["gin"],
                                 self.sg, self.ws.handle, _stream()), "sof_render_bwd", self.ws.handle)

    def reserve(self):
        """Size the workspace for every call (sof_workspace_reserve; synchronises). Two rounds: the
        capacity hints only grow, and every call is sized with the hints of all calls."""
        for _ in range(2 if len(self.calls) > 1 else 1):
            for call in self.calls:
                self.ws.reserve(self.scene_c, call["cams_c"], len(call["cams"]), self.opts_async)
        self._reserved = True
        return self

    def run(self):
        """Eager step: the workspace reserved once, then per call a stream-ordered forward and its
        backward. Check dropped() (or ok()) before using the results."""
        if not getattr(self, "_reserved", False):
            self.reserve()
        self._run_async()

    def _run_async(self):
        L.sof_workspace_clear_dropped(self.ws.handle, _stream())
        for t in self.grads:
            t.zero_()
        for call in self.calls:
            L.check(L.sof_render_fwd(self.scene_c, call["cams_c"], len(call["cams"]), self.opts_async, call["outs_c"],
                                     self.ws.handle, _stream()), "sof_render_fwd", self.ws.handle)
            self._bwd(call, self.opts_async)

    def capture(self, max_retries: int = 4):
        """Capture the step (gradients zeroed, then each call's forward and backward) in a CUDA
        graph through sof_graph_capture, growing the workspace as it asks."""
        self.release()
        cur = torch.cuda.current_stream()
        side = torch.cuda.Stream(cur.device)  # the legacy default stream cannot be captured
        side.wait_stream(cur)
        for _ in range(max_retries):
            rc, g = L.sof_graph_capture(self.scene_c, self.cams_all_c, len(self.cams), self.vpc, self.opts_async,
                                        self.outs_all_c, self.gin_all, self.sg, True, self.ws.handle, side.cuda_stream)
            if rc == L.SOF_ERR_WORKSPACE_TOO_SMALL:
                side.synchronize()
                self.ws.ensure(L.sof_workspace_required(self.ws.handle))
                continue
            L.check(rc, "sof_graph_capture", self.ws.handle)
            cur.wait_stream(side)
            self.graph = g
            return self
        raise L.SOFError(L.SOF_ERR_WORKSPACE_TOO_SMALL, "sof_graph_capture")

    def replay(self):
        if self.graph is None:
            raise RuntimeError("capture() first")
        L.check(L.sof_graph_launch(self.graph, _stream()), "sof_graph_launch", self.ws.handle)

    def release(self):
        if self.graph is not None:
            L.sof_graph_destroy(self.graph)
            self.graph = None

    def __del__(self):
        try:
            self.release()
        except Exception:
            pass

    def stats(self) -> dict:
        """Counters of the last call (the last group); n_dropped covers every call of the step."""
        torch.cuda.synchronize()  # a replay runs on the current stream, not the capture stream
        return self.ws.stats()

    def dropped(self) -> int:
        """Pairs or visible records the step's calls could not hold (the results are invalid if > 0)."""
        return int(self.stats()["n_dropped"])

    def ok(self) -> bool:
        return self.dropped() == 0


class QueryGraph:
    """An opacity query (sof_opacity_query) over fixed points and views, captured in a CUDA graph.

    The Gaussians' tensors and the points are held by reference: a replay reads their current
    values and writes `opacity` and `seen`. capture() runs the query once synchronously, which
    sizes the workspace, then captures it with SOF_QUERY_ASYNC (no host round trip per view). The
    capacities then stay fixed, so check each replay with dropped() (or ok())."""

    def __init__(self, gauss_tensors, cams, points, opts=None, ws: Workspace | None = None):
        from .render import QueryOptions
        means, log_scales, quats, logits = gauss_tensors[:4]
        self.refs = (means, log_scales, quats, logits, points)
        dev = means.device
        self._sh = torch.zeros((means.shape[0], 1, 3), dtype=torch.float32, device=dev)
        self.scene_c = scene_to_c(means, log_scales, quats, logits, self._sh)
        self.scene_c.sh = 0
        self.cams = list(cams)
        self.cams_c = cameras_to_c(self.cams)
        opts = opts or QueryOptions()
        self.opts_sync = dataclasses.replace(opts, async_mode=False).to_c()
        self.opts_async = dataclasses.replace(opts, async_mode=True).to_c()
        if not (points.is_cuda and points.dtype == torch.float32 and points.is_contiguous()):
            raise ValueError("points must be a contiguous float32 CUDA tensor [P,3]")
        self.points = points
        self.n = int(points.shape[0])
        self.opacity = torch.empty(self.n, dtype=torch.float32, device=dev)
        self.seen = torch.empty(self.n, dtype=torch.int32, device=dev)
        self.ws = ws or Workspace(dev)
        self.graph = None

    def _call(self, opts_c):
        return L.sof_opacity_query(self.scene_c, self.cams_c, len(self.cams), self.points.data_ptr(), self.n, opts_c,
                                   self.opacity.data_ptr(), self.seen.data_ptr(), self.ws.handle, _stream())

    def run(self, max_retries: int = 4):
        """The synchronous query (grows the workspace as needed)."""
        if self.ws.buffer is None:
            self.ws.ensure(L.sof_query_workspace_size(self.scene_c, self.cams_c, len(self.cams), self.n,
                                                      self.opts_sync, max(4 * self.scene_c.n, 1 << 16)))
        for _ in range(max_retries):
            rc = self._call(self.opts_sync)
            if rc != L.SOF_ERR_WORKSPACE_TOO_SMALL:
                L.check(rc, "sof_opacity_query", self.ws.handle)
                return self
            self.ws.ensure(L.sof_workspace_required(self.ws.handle))
        raise L.SOFError(L.SOF_ERR_WORKSPACE_TOO_SMALL, "sof_opacity_query")

    def capture(self):
        self.run()
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            L.check(self._call(self.opts_async), "sof_opacity_query", self.ws.handle)
        self.graph = g
        return self

    def replay(self):
        if self.graph is None:
            raise RuntimeError("capture() first")
        self.graph.replay()

    def dropped(self) -> int:
        """Gaussian pairs the captured capacities could not hold (the results are invalid if > 0)."""
        torch.cuda.synchronize()
        return int(self.ws.stats()["n_dropped"])

    def ok(self) -> bool:
        return self.dropped() == 0


class InputPipeline:
    """Double-buffered upload of per-step inputs from pinned host memory.

    The copies run on a side stream into two device buffer sets, so the upload for step i + 1
    overlaps the render of step i on the compute stream. upload(host, slot) queues a copy into
    buffer set `slot` once the compute stream has released it; acquire(slot) makes the compute
    stream wait for that copy and returns the buffers; release(slot) marks them free again after
    the work queued so far on the compute stream.
    """

    def __init__(self, like, device=None):
        device = device or like[0].device
        self.bufs = [[torch.empty_like(t, device=device) for t in like] for _ in range(2)]
        self.copy_stream = torch.cuda.Stream(device)
        self.ready = [torch.cuda.Event() for _ in range(2)]
        self.free = [torch.cuda.Event() for _ in range(2)]

    def upload(self, host, slot: int, after: torch.cuda.Stream | None = None):
        """Queue host -> bufs[slot]. `after`: a stream whose queued work the copy also waits for."""
        if len(host) != len(self.bufs[slot]) or any(h.shape != d.shape or h.dtype != d.dtype
                                                     for h, d in zip(host, self.bufs[slot])):
            raise ValueError("host inputs do not match the buffers")
        if not all(h.is_pinned() for h in host):
            raise ValueError("host inputs must be in pinned memory")
        cs = self.copy_stream
        if after is not None:
            cs.wait_stream(after)
        cs.wait_event(self.free[slot])  # no-op before the first release
        with torch.cuda.stream(cs):
            for h, d in zip(host, self.bufs[slot]):
                d.copy_(h, non_blocking=True)
            self.ready[slot].record(cs)

    def acquire(self, slot: int, stream: torch.cuda.Stream | None = None):
        (stream or torch.cuda.current_stream()).wait_event(self.ready[slot])
        return self.bufs[slot]

    def release(self, slot: int, stream: torch.cuda.Stream | None = None):
        self.free[slot].record(stream or torch.cuda.current_stream())
