"""sof_render_fwd_noalloc: the forward render for callers that cannot allocate device memory.

It must produce what sof_render_fwd produces with a caller-bound workspace, call after call (the
fixed scratch array is shared and keeps the previous call's contents), and refuse scenes that do not
fit its fixed scratch with a clear status instead of allocating. Collected last on purpose (file
name), so that a run stopping at the first failure has already run every other test; it passes
both alone in a fresh process and after the other tests.
"""
import gc
import math

import numpy as np
import pytest
import torch

from paper_2506_19139_gb300 import _lib as L
from paper_2506_19139_gb300 import render as R
from paper_2506_19139_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2506_19139_gb300 import build
    build.build()


def _inputs(scene, cams):
    ts = R.scene_tensors(scene)
    return ts, R.scene_to_c(*ts), R.cameras_to_c(cams)


def _reference(ts, scene_c, cams_c, cams, opts_c):
    outs = R.alloc_outputs(cams, ts[0].device)
    R.render_forward_raw(scene_c, cams_c, len(cams), opts_c, outs, R.Workspace())
    return outs


def _noalloc(scene_c, cams_c, cams, opts_c):
    outs = R.alloc_outputs(cams, "cuda")
    rc, req = L.sof_render_fwd_noalloc(scene_c, cams_c, len(cams), opts_c, R._out_c(outs),
                                       torch.cuda.current_stream().cuda_stream)
    return rc, req, outs


def _same(a, b):
    torch.cuda.synchronize()
    for k in ("color", "depth", "exact_depth", "normal", "opacity"):
        assert (a[k] - b[k]).abs().max().item() <= 1e-5, k
    assert torch.equal(a["n_contrib"], b["n_contrib"])


def test_noalloc_matches_workspace_path_on_consecutive_calls():
    opts_c = R.RenderOptions().to_c()
    scene_a, cams_a = syn.tiny_forward(0)
    scene_b = syn.uniform_box_scene(1500, 8, 1.0, (0.01, 0.2), (0.1, 0.99), 1)
    cams_b = [syn.look_at((0.5, -0.3, 3.5), (0.0, 0.1, 0.0), 75, 45, 55.0),
              syn.look_at((-3.0, 0.5, 2.0), (0.0, 0.0, 0.0), 40, 56, 60.0)]
    for scene, cams in ((scene_a, cams_a), (scene_b, cams_b), (scene_a, cams_a)):
        ts, scene_c, cams_c = _inputs(scene, cams)
        rc, req, got = _noalloc(scene_c, cams_c, cams, opts_c)
        assert rc == L.SOF_OK, L.error_string(rc)
        _same(got, _reference(ts, scene_c, cams_c, cams, opts_c))
        assert float(got["opacity"].max()) > 0.1


def test_noalloc_allocates_nothing():
    """After a first call on the device (which looks up the array's address), further calls leave
    both torch's allocator and the device's free memory unchanged."""
    opts_c = R.RenderOptions().to_c()
    scene, cams = syn.tiny_forward(0)
    ts, scene_c, cams_c = _inputs(scene, cams)
    outs = R.alloc_outputs(cams, "cuda")
    stream = torch.cuda.current_stream().cuda_stream
    rc, _ = L.sof_render_fwd_noalloc(scene_c, cams_c, 1, opts_c, R._out_c(outs), stream)
    assert rc == L.SOF_OK
    # earlier tests' tensors freed by the garbage collector meanwhile would lower the counts: collect
    # them first, and require that nothing grows
    gc.collect()
    torch.cuda.synchronize()
    alloc0, free0 = torch.cuda.memory_allocated(), torch.cuda.mem_get_info()[0]
    for _ in range(3):
        rc, _ = L.sof_render_fwd_noalloc(scene_c, cams_c, 1, opts_c, R._out_c(outs), stream)
        assert rc == L.SOF_OK
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() <= alloc0
    assert torch.cuda.mem_get_info()[0] >= free0


@pytest.mark.parametrize("flags", [0, L.SOF_FLAG_ASYNC])
def test_noalloc_rejects_scenes_beyond_its_fixed_scratch(flags):
    """Also when the caller asks for a stream-ordered forward: the no-allocation call is always
    checked, so a scene that does not fit is refused, never rendered with pairs dropped."""
    scene = syn.uniform_box_scene(200_000, 3, 1.0, (0.01, 0.1), (0.1, 0.99), 0)
    cams = [syn.look_at((0.0, 0.0, 4.0), (0.0, 0.0, 0.0), 256, 256, 60.0)]
    ts, scene_c, cams_c = _inputs(scene, cams)
    o = R.RenderOptions().to_c()
    o.flags = flags
    rc, req, _ = _noalloc(scene_c, cams_c, cams, o)
    assert rc == L.SOF_ERR_WORKSPACE_TOO_SMALL
    assert req > (24 << 20)
    assert L.sof_noalloc_last_error() == "workspace too small"
    # a following small call still works
    scene_a, cams_a = syn.tiny_forward(0)
    ts, scene_c, cams_c = _inputs(scene_a, cams_a)
    rc, _, got = _noalloc(scene_c, cams_c, cams_a, R.RenderOptions().to_c())
    assert rc == L.SOF_OK
    _same(got, _reference(ts, scene_c, cams_c, cams_a, R.RenderOptions().to_c()))


def test_noalloc_empty_and_fully_culled_scenes():
    """No Gaussians, and Gaussians all behind the camera: the call succeeds with the background
    image, like the workspace path."""
    scene_a, cams = syn.tiny_forward(0)
    empty = scene_a.subset(np.arange(0))
    behind = scene_a.subset(np.arange(200))
    behind.means[:, 2] += 10.0  # the camera at z = 4 looks toward -z: all of them behind it
    opts = R.RenderOptions(bg=(0.2, 0.4, 0.6))
    for scene in (empty, behind):
        ts, scene_c, cams_c = _inputs(scene, cams)
        rc, _, got = _noalloc(scene_c, cams_c, cams, opts.to_c())
        assert rc == L.SOF_OK
        _same(got, _reference(ts, scene_c, cams_c, cams, opts.to_c()))
        img = R.view_images(got, cams)[0]
        assert torch.allclose(img["color"], torch.tensor([0.2, 0.4, 0.6], device="cuda")[:, None, None])
        assert torch.all(img["opacity"] == 0)
