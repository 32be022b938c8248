"""PyTorch front end of the compositing core: device memory, streams and autograd glue around the
C-ABI calls (sof_render_fwd / sof_render_bwd / sof_opacity_query). Every step of the computation
runs in the CUDA library; this module only allocates tensors and passes pointers."""
from __future__ import annotations

import ctypes as C
import dataclasses
from typing import Sequence

import torch

from . import _lib as L


@dataclasses.dataclass
class RenderOptions:
    near_plane: float = 0.2
    t_stop: float = 1e-4
    bg: tuple = (0.0, 0.0, 0.0)
    tile: int = 16
    chunk: int = 64
    reorder_k: int = 16
    median_depth: bool = False
    replay_cap: int = 256  # hits per pixel the forward records for the backward; -1: none
    # stream-ordered forward (the library's default: capacities from the bound workspace, excess
    # dropped and counted) instead of the checked one, which reads the pair bound back and grows
    # the workspace (SOF_FLAG_CHECKED)
    async_mode: bool = False
    sort_prefix: int = 0  # keys per tile sorted up front: 0 = library default, -1 = whole lists
    approx_order: bool = False  # opt-in approximate per-pixel order (SOF_FLAG_APPROX_ORDER)
    losses: bool = False  # also the distortion and extent loss channels
    opacity_at_depth: bool = False  # also the opacity field at the exact depth (needs recorded hits)

    def to_c(self) -> L.sof_render_opts:
        o = L.sof_render_opts()
        o.near_plane = self.near_plane
        o.t_stop = self.t_stop
        for i in range(3):
            o.bg[i] = float(self.bg[i])
        o.tile, o.chunk, o.reorder_k = self.tile, self.chunk, self.reorder_k
        o.flags = ((L.SOF_FLAG_MEDIAN_DEPTH if self.median_depth else 0) | (0 if self.async_mode else L.SOF_FLAG_CHECKED) |
                   (L.SOF_FLAG_APPROX_ORDER if self.approx_order else 0))
        o.replay_cap = self.replay_cap
        o.sort_prefix = self.sort_prefix
        return o


@dataclasses.dataclass
class QueryOptions:
    near_plane: float = 0.2
    t_stop_query: float = 0.0
    tile: int = 16
    level_set: bool = False  # only O > 0.5 is exact (SOF_QUERY_LEVEL_SET)
    async_mode: bool = False  # no host round trip per view: capturable in a CUDA graph (SOF_QUERY_ASYNC)
    prepared: bool = False  # use the views prepare_query() left resident (SOF_QUERY_PREPARED)

    def to_c(self) -> L.sof_query_opts:
        o = L.sof_query_opts()
        o.near_plane, o.t_stop_query, o.tile = self.near_plane, self.t_stop_query, self.tile
        o.flags = ((L.SOF_QUERY_LEVEL_SET if self.level_set else 0) | (L.SOF_QUERY_ASYNC if self.async_mode else 0) |
                   (L.SOF_QUERY_PREPARED if self.prepared else 0))
        return o


def cameras_to_c(cams) -> "C.Array":
    arr = (L.sof_camera * len(cams))()
    for i, c in enumerate(cams):
        w2c = c.world_to_cam.reshape(-1)
        for j in range(12):
            arr[i].world_to_cam[j] = float(w2c[j])
        arr[i].fx, arr[i].fy, arr[i].cx, arr[i].cy = float(c.fx), float(c.fy), float(c.cx), float(c.cy)
        arr[i].width, arr[i].height = int(c.width), int(c.height)
    return arr


def _ptr(t):
    return 0 if t is None else t.data_ptr()


def scene_to_c(means, log_scales, quats, opacity_logits, sh) -> L.sof_scene:
    for name, t in (("means", means), ("log_scales", log_scales), ("quats", quats),
                    ("opacity_logits", opacity_logits), ("sh", sh)):
        if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
            raise ValueError(f"{name} must be a contiguous float32 CUDA tensor")
    k = sh.shape[1]
    deg = {1: 0, 4: 1, 9: 2, 16: 3}[k]
    s = L.sof_scene()
    s.means, s.log_scales, s.quats = means.data_ptr(), log_scales.data_ptr(), quats.data_ptr()
    s.opacity_logits, s.sh = opacity_logits.data_ptr(), sh.data_ptr()
    s.n, s.sh_degree = means.shape[0], deg
    return s


class Workspace:
    """Caller-owned device scratch bound to a library workspace handle; grows on demand."""

    def __init__(self, device="cuda", initial_bytes: int = 0):
        self.handle = L.sof_workspace_create()
        self.device = torch.device(device)
        self.buffer = None
        # forwards run on this workspace: a backward must follow its own forward (the workspace
        # holds the sorted lists of the last forward only)
        self.generation = 0
        if initial_bytes:
            self.ensure(initial_bytes)

    def reserve(self, scene_c, cams_c, n_views, opts_c, max_retries: int = 4) -> int:
        """Grow the workspace to what a stream-ordered render of this scene and these views needs
        (sof_workspace_reserve; synchronises). Returns the bytes bound."""
        if self.buffer is None:
            self.ensure(L.sof_render_workspace_size(scene_c, cams_c, n_views, opts_c, 1 << 16))
        for _ in range(max_retries):
            rc, need = L.sof_workspace_reserve(self.handle, scene_c, cams_c, n_views, opts_c, _stream())
            if rc == L.SOF_ERR_WORKSPACE_TOO_SMALL:
                self.ensure(L.sof_workspace_required(self.handle))
                continue
            L.check(rc, "sof_workspace_reserve", self.handle)
            self.ensure(need)
            return need
        raise L.SOFError(L.SOF_ERR_WORKSPACE_TOO_SMALL, "sof_workspace_reserve")

    def ensure(self, nbytes: int):
        if self.buffer is None or self.buffer.numel() < nbytes:
            self.buffer = torch.empty(int(nbytes) + 256, dtype=torch.uint8, device=self.device)
            base = (self.buffer.data_ptr() + 255) // 256 * 256
            L.sof_workspace_bind(self.handle, base, int(nbytes))

    def stats(self) -> dict:
        return L.sof_workspace_stats(self.handle)

    def __del__(self):
        try:
            if getattr(self, "handle", None) is not None:
                L.sof_workspace_destroy(self.handle)
        except Exception:
            pass


def _stream():
    return torch.cuda.current_stream().cuda_stream


def alloc_outputs(cams, device, median=False, losses=False, opa=False):
    npx = sum(int(c.width) * int(c.height) for c in cams)
    f = dict(dtype=torch.float32, device=device)
    return {
        "color": torch.empty(3 * npx, **f), "depth": torch.empty(npx, **f), "exact_depth": torch.empty(npx, **f),
        "median_depth": torch.empty(npx, **f) if median else None, "normal": torch.empty(3 * npx, **f),
        "opacity": torch.empty(npx, **f), "n_contrib": torch.empty(npx, dtype=torch.int32, device=device),
        "distortion": torch.empty(npx, **f) if losses else None, "extent": torch.empty(npx, **f) if losses else None,
        "opacity_at_depth": torch.empty(npx, **f) if opa else None,
    }


def _out_c(o) -> L.sof_render_out:
    c = L.sof_render_out()
    c.color, c.depth, c.exact_depth = _ptr(o["color"]), _ptr(o["depth"]), _ptr(o["exact_depth"])
    c.median_depth, c.normal, c.opacity = _ptr(o["median_depth"]), _ptr(o["normal"]), _ptr(o["opacity"])
    c.n_contrib = _ptr(o["n_contrib"])
    c.distortion, c.extent = _ptr(o.get("distortion")), _ptr(o.get("extent"))
    c.opacity_at_depth = _ptr(o.get("opacity_at_depth"))
    return c


def render_forward_raw(scene_c, cams_c, n_views, opts_c, outs, ws: Workspace, max_retries: int = 4) -> int:
    """sof_render_fwd with workspace growth on SOF_ERR_WORKSPACE_TOO_SMALL. Returns the status."""
    oc = _out_c(outs)
    ws.generation += 1
    if ws.buffer is None:
        ws.ensure(L.sof_render_workspace_size(scene_c, cams_c, n_views, opts_c, max(4 * scene_c.n * n_views, 1 << 16)))
    for _ in range(max_retries):
        rc = L.sof_render_fwd(scene_c, cams_c, n_views, opts_c, oc, ws.handle, _stream())
        if rc != L.SOF_ERR_WORKSPACE_TOO_SMALL:
            return L.check(rc, "sof_render_fwd", ws.handle)
        ws.ensure(L.sof_workspace_required(ws.handle))
    raise L.SOFError(L.SOF_ERR_WORKSPACE_TOO_SMALL, "sof_render_fwd")


def split_views(flat, cams, channels):
    out, off = [], 0
    for c in cams:
        n = channels * c.width * c.height
        v = flat[off:off + n]
        out.append(v.view(channels, c.height, c.width) if channels > 1 else v.view(c.height, c.width))
        off += n
    return out


class _SOFRenderFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, means, log_scales, quats, opacity_logits, sh, cams, opts, ws):
        scene_c = scene_to_c(means, log_scales, quats, opacity_logits, sh)
        cams_c = cameras_to_c(cams)
        opts_c = opts.to_c()
        outs = alloc_outputs(cams, means.device, opts.median_depth, opts.losses, opts.opacity_at_depth)
        render_forward_raw(scene_c, cams_c, len(cams), opts_c, outs, ws)
        ctx.save_for_backward(means, log_scales, quats, opacity_logits, sh)
        ctx.cams, ctx.opts, ctx.ws, ctx.outs = cams, opts, ws, outs
        ctx.generation = ws.generation
        ctx.mark_non_differentiable(outs["n_contrib"])
        empty = torch.zeros(0, device=means.device)
        med = outs["median_depth"] if outs["median_depth"] is not None else empty
        dist = outs["distortion"] if outs["distortion"] is not None else empty
        ext = outs["extent"] if outs["extent"] is not None else empty
        opa = outs["opacity_at_depth"] if outs["opacity_at_depth"] is not None else empty
        return (outs["color"], outs["depth"], outs["exact_depth"], med, outs["normal"], outs["opacity"],
                outs["n_contrib"], dist, ext, opa)

    @staticmethod
    def backward(ctx, g_color, g_depth, g_exact, g_med, g_normal, g_opacity, _g_n, g_dist, g_ext, g_opa):
        means, log_scales, quats, opacity_logits, sh = ctx.saved_tensors
        if ctx.ws.generation != ctx.generation:
            raise RuntimeError("the workspace rendered another forward after this one: its backward needs this "
                               "forward's sorted lists (give each render() that will be differentiated its own "
                               "Workspace)")
        scene_c = scene_to_c(means, log_scales, quats, opacity_logits, sh)
        cams_c = cameras_to_c(ctx.cams)
        grads = [torch.zeros_like(t) for t in (means, log_scales, quats, opacity_logits, sh)]
        gin = L.sof_render_grad_in()

        def cp(g):
            return 0 if g is None else g.contiguous().data_ptr()
        keep = [None if g is None else g.contiguous()
                for g in (g_color, g_depth, g_exact, g_med, g_normal, g_opacity, g_dist, g_ext, g_opa)]
        gin.d_color, gin.d_depth, gin.d_exact_depth = cp(keep[0]), cp(keep[1]), cp(keep[2])
        gin.d_median_depth = cp(keep[3]) if ctx.opts.median_depth else 0
        gin.d_normal, gin.d_opacity = cp(keep[4]), cp(keep[5])
        if ctx.opts.losses:
            gin.d_distortion, gin.d_extent = cp(keep[6]), cp(keep[7])
        if ctx.opts.opacity_at_depth:
            gin.d_opacity_at_depth = cp(keep[8])
        sg = L.sof_scene_grad()
        sg.d_means, sg.d_log_scales, sg.d_quats = grads[0].data_ptr(), grads[1].data_ptr(), grads[2].data_ptr()
        sg.d_opacity_logits, sg.d_sh = grads[3].data_ptr(), grads[4].data_ptr()
        L.check(L.sof_render_bwd(scene_c, cams_c, len(ctx.cams), ctx.opts.to_c(), _out_c(ctx.outs), gin, sg,
                                 ctx.ws.handle, _stream()), "sof_render_bwd", ctx.ws.handle)
        return (*grads, None, None, None)


def render(means, log_scales, quats, opacity_logits, sh, cams: Sequence, opts: RenderOptions | None = None,
           ws: Workspace | None = None):
    """Differentiable exact-order render of one or more views. Returns a dict with flat per-view
    packed tensors and per-view image lists ('images')."""
    opts = opts or RenderOptions()
    if not (torch.is_grad_enabled() and any(t.requires_grad for t in (means, log_scales, quats, opacity_logits, sh))) \
            and not opts.opacity_at_depth:
        opts = dataclasses.replace(opts, replay_cap=-1)  # no backward follows: record nothing
    ws = ws or Workspace(means.device)
    color, depth, exact, med, normal, opacity, n_contrib, dist, ext, opa = _SOFRenderFn.apply(
        means, log_scales, quats, opacity_logits, sh, list(cams), opts, ws)
    return {"color": color, "depth": depth, "exact_depth": exact, "median_depth": med if opts.median_depth else None,
            "normal": normal, "opacity": opacity, "n_contrib": n_contrib, "workspace": ws,
            "distortion": dist if opts.losses else None, "extent": ext if opts.losses else None,
            "opacity_at_depth": opa if opts.opacity_at_depth else None}


def view_images(res, cams):
    """Per-view [3,H,W] / [H,W] views of the packed outputs of render()."""
    out = []
    imgs = {k: split_views(res[k], cams, 3 if k in ("color", "normal") else 1)
            for k in ("color", "depth", "exact_depth", "normal", "opacity", "n_contrib")}
    for k in ("distortion", "extent", "opacity_at_depth"):
        if res.get(k) is not None:
            imgs[k] = split_views(res[k], cams, 1)
    if res.get("median_depth") is not None:
        imgs["median_depth"] = split_views(res["median_depth"], cams, 1)
    for i in range(len(cams)):
        out.append({k: v[i] for k, v in imgs.items()})
    return out


def scene_tensors(scene, device="cuda", requires_grad=False):
    """Upload a synthetic.Scene to the device as contiguous float32 tensors."""
    ts = [torch.as_tensor(x, device=device).float().contiguous() for x in
          (scene.means, scene.log_scales, scene.quats, scene.opacity_logits, scene.sh)]
    if requires_grad:
        for t in ts:
            t.requires_grad_(True)
    return ts


def opacity_query(means, log_scales, quats, opacity_logits, cams: Sequence, points, opts: QueryOptions | None = None,
                  ws: Workspace | None = None, max_retries: int = 4):
    """Opacity field at points, min over the views that see each point (sof_opacity_query).
    Returns (opacity [P] float32, seen_count [P] int32) on the points' device."""
    opts = opts or QueryOptions()
    ws = ws or Workspace(means.device)
    dummy_sh = torch.zeros((means.shape[0], 1, 3), dtype=torch.float32, device=means.device)
    scene_c = scene_to_c(means, log_scales, quats, opacity_logits, dummy_sh)
    scene_c.sh = 0
    cams_c = cameras_to_c(cams)
    opts_c = opts.to_c()
    pts = points.contiguous()
    P = pts.shape[0]
    out = torch.empty(P, dtype=torch.float32, device=pts.device)
    seen = torch.empty(P, dtype=torch.int32, device=pts.device)
    if ws.buffer is None:
        ws.ensure(L.sof_query_workspace_size(scene_c, cams_c, len(cams), P, opts_c, max(4 * scene_c.n, 1 << 16)))
    for _ in range(max_retries):
        rc = L.sof_opacity_query(scene_c, cams_c, len(cams), pts.data_ptr(), P, opts_c, out.data_ptr(),
                                 seen.data_ptr(), ws.handle, _stream())
        if rc != L.SOF_ERR_WORKSPACE_TOO_SMALL:
            L.check(rc, "sof_opacity_query", ws.handle)
            return out, seen
        ws.ensure(L.sof_workspace_required(ws.handle))
    raise L.SOFError(L.SOF_ERR_WORKSPACE_TOO_SMALL, "sof_opacity_query")


def level_set_bisect(means, log_scales, quats, opacity_logits, cams: Sequence, inside, outside, iterations: int = 8,
                     opts: QueryOptions | None = None, ws: Workspace | None = None, max_retries: int = 4):
    """Bisection for the 0.5 level set of O along edges (sof_level_set_bisect): `inside` [E,3] has
    O > 0.5, `outside` [E,3] has O <= 0.5. Both are updated in place and returned; the crossing lies
    between them, 2^-iterations of the original edge apart."""
    opts = dataclasses.replace(opts or QueryOptions(), level_set=True)
    ws = ws or Workspace(means.device)
    dummy_sh = torch.zeros((means.shape[0], 1, 3), dtype=torch.float32, device=means.device)
    scene_c = scene_to_c(means, log_scales, quats, opacity_logits, dummy_sh)
    scene_c.sh = 0
    cams_c = cameras_to_c(cams)
    opts_c = opts.to_c()
    for t in (inside, outside):
        if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous() and t.dim() == 2 and t.shape[1] == 3):
            raise ValueError("inside / outside must be contiguous float32 CUDA tensors [E,3]")
    E = inside.shape[0]
    if ws.buffer is None:
        ws.ensure(L.sof_query_workspace_size(scene_c, cams_c, len(cams), E, opts_c, max(4 * scene_c.n, 1 << 16))
                  + 16 * E + 1024)
    for _ in range(max_retries):
        # a too-small workspace is reported before any endpoint moves
        rc = L.sof_level_set_bisect(scene_c, cams_c, len(cams), inside.data_ptr(), outside.data_ptr(), E, iterations,
                                    opts_c, ws.handle, _stream())
        if rc != L.SOF_ERR_WORKSPACE_TOO_SMALL:
            L.check(rc, "sof_level_set_bisect", ws.handle)
            return inside, outside
        ws.ensure(L.sof_workspace_required(ws.handle))
    raise L.SOFError(L.SOF_ERR_WORKSPACE_TOO_SMALL, "sof_level_set_bisect")


def prepare_query(means, log_scales, quats, opacity_logits, cams: Sequence, max_points: int,
                  opts: QueryOptions | None = None, ws: Workspace | None = None, max_retries: int = 4) -> Workspace:
    """sof_query_prepare: every view's Gaussian lists built once and kept resident in the workspace
    (grown as the library asks, with room for queries of up to max_points points); later
    opacity_query / level_set_bisect calls with QueryOptions(prepared=True) on this workspace do
    only the points' work."""
    opts = opts or QueryOptions()
    ws = ws or Workspace(means.device)
    dummy_sh = torch.zeros((means.shape[0], 1, 3), dtype=torch.float32, device=means.device)
    scene_c = scene_to_c(means, log_scales, quats, opacity_logits, dummy_sh)
    scene_c.sh = 0
    cams_c = cameras_to_c(cams)
    opts_c = opts.to_c()
    if ws.buffer is None:
        ws.ensure(1 << 20)
    for _ in range(max_retries):
        rc = L.sof_query_prepare(scene_c, cams_c, len(cams), int(max_points), opts_c, ws.handle, _stream())
        if rc != L.SOF_ERR_WORKSPACE_TOO_SMALL:
            L.check(rc, "sof_query_prepare", ws.handle)
            return ws
        ws.ensure(L.sof_workspace_required(ws.handle))
    raise L.SOFError(L.SOF_ERR_WORKSPACE_TOO_SMALL, "sof_query_prepare")
