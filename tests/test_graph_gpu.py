"""The batched path: many views in one call, the CUDA-graph-captured training step and the
autotuner.

- Rendering views together (one preprocess, one binning pass, one tile sort and one composite
  launch over all views' tiles) gives bit-identical images to rendering them one call at a time.
- A forward + backward step captured in a CUDA graph (forward without its host round trip) replays
  to the eager results: images bit-identical, gradients equal up to the order of float atomics;
  after the parameters change in place, a replay equals a fresh eager step.
- A replay whose scene outgrows the captured capacities reports the dropped pairs instead of
  returning a silently wrong image.
- The autotuner returns an instantiated (tile, chunk, reorder_k); every candidate renders the same
  image.
- Through the C-ABI alone (raw pointers, no Python step object): sof_autotune, then
  sof_graph_capture and sof_graph_launch of the tuned step give the images of sof_render_fwd and
  the gradients of sof_render_bwd.
- A backward must follow its own forward: after a second forward on the workspace, the first one's
  backward is refused (other cameras or other outputs), in C and in the autograd front end.
"""
import math

import numpy as np
import pytest
import torch

from paper_2506_19139_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2506_19139_gb300 import build
    build.build()


def _cams():
    return [syn.look_at((3.5 * math.sin(a), 0.3, 3.5 * math.cos(a)), (0.0, 0.0, 0.0), w, h, 60.0)
            for a, (w, h) in zip((0.0, 1.3, 2.9, 4.4), ((96, 64), (50, 77), (128, 96), (33, 40)))]


def _images(res, cams):
    from paper_2506_19139_gb300 import render as R
    return [{k: v.detach().cpu().numpy() for k, v in im.items() if v is not None} for im in R.view_images(res, cams)]


@pytest.mark.parametrize("tile", [16, 32, 8])
def test_batched_views_equal_single_view_calls(tile):
    from paper_2506_19139_gb300 import render as R
    scene = syn.uniform_box_scene(3000, 7, 1.0, (0.02, 0.2), (0.1, 0.99), 2)
    cams = _cams()
    ts = R.scene_tensors(scene)
    o = R.RenderOptions(tile=tile, reorder_k=8 if tile == 32 else 16)
    with torch.no_grad():
        batched = _images(R.render(*ts, cams, o), cams)
        for v, cam in enumerate(cams):
            single = _images(R.render(*ts, [cam], o), [cam])[0]
            for k in single:
                np.testing.assert_array_equal(batched[v][k], single[k], err_msg=f"view {v} {k}")


def _step(scene, cams, seed=0, views_per_call=None):
    from paper_2506_19139_gb300 import render as R
    from paper_2506_19139_gb300.graph import RenderStep
    ts = R.scene_tensors(scene)
    npx = sum(c.width * c.height for c in cams)
    g = torch.Generator(device="cuda").manual_seed(seed)
    gin = {"color": torch.randn(3 * npx, device="cuda", generator=g), "depth": torch.randn(npx, device="cuda", generator=g),
           "opacity": torch.randn(npx, device="cuda", generator=g), "normal": torch.randn(3 * npx, device="cuda", generator=g)}
    return ts, gin, RenderStep(ts, cams, R.RenderOptions(), gin, views_per_call=views_per_call)


def _snapshot(step):
    torch.cuda.synchronize()
    return ({k: v.clone() for k, v in step.outs.items() if v is not None}, [g.clone() for g in step.grads])


def _same(a, b, label):
    outs_a, grads_a = a
    outs_b, grads_b = b
    for k in outs_a:
        assert torch.equal(outs_a[k], outs_b[k]), f"{label}: {k}"
    for x, y in zip(grads_a, grads_b):
        scale = float(y.abs().max()) + 1e-30
        assert float((x - y).abs().max()) <= 1e-5 * scale, label


@pytest.mark.parametrize("views_per_call", [None, 1, 3])
def test_graph_replay_matches_eager_and_follows_parameter_updates(views_per_call):
    """All four views in one call, one call per view, and calls of three views (one workspace,
    gradients summed over the calls)."""
    from paper_2506_19139_gb300.graph import RenderStep
    scene = syn.uniform_box_scene(3000, 8, 1.0, (0.02, 0.2), (0.1, 0.99), 2)
    cams = _cams()
    ts, gin, step = _step(scene, cams, views_per_call=views_per_call)
    step.run()
    eager = _snapshot(step)
    step.capture()
    step.replay()
    assert step.ok()
    _same(_snapshot(step), eager, "replay")
    # move the Gaussians in place: the graph reads the same tensors
    with torch.no_grad():
        ts[0].add_(0.01 * torch.randn_like(ts[0]))
        ts[3].add_(0.1)
    step.replay()
    assert step.ok()
    fresh = RenderStep(ts, cams, step.opts, gin)  # all views in one eager call
    fresh.run()
    _same(_snapshot(step), _snapshot(fresh), "after update")


def test_replay_reports_pairs_beyond_its_capacity():
    """Calls of two views: the overflow of either call is reported for the whole step."""
    scene = syn.uniform_box_scene(3000, 9, 1.0, (0.01, 0.05), (0.1, 0.99), 0)
    cams = _cams()
    ts, gin, step = _step(scene, cams, views_per_call=2)
    step.capture()
    step.replay()
    assert step.ok()
    big = syn.uniform_box_scene(3000, 9, 1.0, (0.2, 0.6), (0.1, 0.99), 0)
    with torch.no_grad():
        ts[1].copy_(torch.as_tensor(big.log_scales, device="cuda"))
    step.replay()
    assert step.dropped() > 0


def test_autotune_returns_an_instantiated_pair_with_identical_images():
    from paper_2506_19139_gb300 import autotune, render as R
    scene = syn.uniform_box_scene(2000, 10, 1.0, (0.02, 0.3), (0.1, 0.99), 1)
    cams = _cams()[:2]
    ts = R.scene_tensors(scene)
    best, times = autotune.tune(ts, cams, reps=1)
    assert (best.tile, best.chunk, best.reorder_k) in autotune.candidates()
    assert set(times) == set(autotune.candidates())
    with torch.no_grad():
        ref = _images(R.render(*ts, cams), cams)
        for tl, ch, k in autotune.candidates():
            got = _images(R.render(*ts, cams, R.RenderOptions(tile=tl, chunk=ch, reorder_k=k)), cams)
            for v in range(len(cams)):
                for key in ref[v]:
                    np.testing.assert_array_equal(got[v][key], ref[v][key], err_msg=f"{tl},{ch},{k} view {v} {key}")


def test_input_pipeline_uploads_each_step_before_its_render():
    """Steps fed by graph.InputPipeline (uploads on a side stream, two buffer sets) render what the
    same inputs render when resident: each step sees its own upload, never the other buffer's."""
    from paper_2506_19139_gb300 import render as R
    from paper_2506_19139_gb300.graph import InputPipeline
    cams = _cams()[:2]
    scenes = [syn.uniform_box_scene(2000, s, 1.0, (0.02, 0.2), (0.1, 0.99), 2) for s in (3, 4, 5)]
    want = []
    with torch.no_grad():
        for sc in scenes:
            want.append(_images(R.render(*R.scene_tensors(sc), cams, R.RenderOptions()), cams))
    hosts = [[t.cpu().pin_memory() for t in R.scene_tensors(sc)] for sc in scenes]
    pipe = InputPipeline(R.scene_tensors(scenes[0]))
    stream = torch.cuda.current_stream()
    got = []
    pipe.upload(hosts[0], 0, after=stream)
    with torch.no_grad():
        for i in range(len(scenes)):
            s = i & 1
            if i + 1 < len(scenes):
                pipe.upload(hosts[i + 1], s ^ 1)
            bufs = pipe.acquire(s, stream)
            got.append(_images(R.render(*bufs, cams, R.RenderOptions()), cams))
            pipe.release(s, stream)
    for i in range(len(scenes)):
        for v in range(len(cams)):
            for k in want[i][v]:
                np.testing.assert_array_equal(got[i][v][k], want[i][v][k], err_msg=f"step {i} view {v} {k}")
    with pytest.raises(ValueError):
        pipe.upload([t.cpu() for t in R.scene_tensors(scenes[0])], 0)


def test_c_abi_tune_capture_replay_matches_fwd_bwd(tmp_path):
    """tune -> capture -> replay on raw device pointers, against separate sof_render_fwd /
    sof_render_bwd calls with the tuned options."""
    from paper_2506_19139_gb300 import _lib as L
    from paper_2506_19139_gb300 import render as R
    scene = syn.uniform_box_scene(2500, 12, 1.0, (0.02, 0.25), (0.1, 0.99), 2)
    cams = _cams()
    ts = R.scene_tensors(scene)
    scene_c, cams_c = R.scene_to_c(*ts), R.cameras_to_c(cams)
    npx = sum(c.width * c.height for c in cams)
    g = torch.Generator(device="cuda").manual_seed(3)
    d_color = torch.randn(3 * npx, device="cuda", generator=g)
    d_opacity = torch.randn(npx, device="cuda", generator=g)
    gin = L.sof_render_grad_in()
    gin.d_color, gin.d_opacity = d_color.data_ptr(), d_opacity.data_ptr()

    def buffers():
        outs = R.alloc_outputs(cams, "cuda")
        grads = [torch.zeros_like(t) for t in ts]
        sg = L.sof_scene_grad()
        sg.d_means, sg.d_log_scales, sg.d_quats = grads[0].data_ptr(), grads[1].data_ptr(), grads[2].data_ptr()
        sg.d_opacity_logits, sg.d_sh = grads[3].data_ptr(), grads[4].data_ptr()
        return outs, grads, sg

    ws = R.Workspace()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    base = R.RenderOptions(async_mode=True).to_c()
    outs, grads, sg = buffers()
    cache = str(tmp_path / "tune.txt")
    ws.ensure(1 << 20)
    for _ in range(4):
        rc, best, ms = L.sof_autotune(scene_c, cams_c, len(cams), 2, base, R._out_c(outs), gin, sg, 1, cache,
                                      ws.handle, side.cuda_stream)
        if rc != L.SOF_ERR_WORKSPACE_TOO_SMALL:
            break
        ws.ensure(L.sof_workspace_required(ws.handle))
    assert rc == L.SOF_OK, L.error_string(rc)
    assert (best.tile, best.chunk, best.reorder_k) in [L.sof_autotune_candidate(i)
                                                       for i in range(L.SOF_AUTOTUNE_CANDIDATES)]
    assert min(m for m in ms if m >= 0) > 0
    # the cached answer comes back without timing
    rc2, best2, ms2 = L.sof_autotune(scene_c, cams_c, len(cams), 2, base, R._out_c(outs), gin, sg, 1, cache,
                                     ws.handle, side.cuda_stream)
    assert rc2 == L.SOF_OK and (best2.tile, best2.chunk, best2.reorder_k) == (best.tile, best.chunk, best.reorder_k)
    outs, grads, sg = buffers()
    for _ in range(4):
        rc, graph = L.sof_graph_capture(scene_c, cams_c, len(cams), 2, best, R._out_c(outs), gin, sg, True,
                                        ws.handle, side.cuda_stream)
        if rc != L.SOF_ERR_WORKSPACE_TOO_SMALL:
            break
        ws.ensure(L.sof_workspace_required(ws.handle))
    assert rc == L.SOF_OK, L.error_string(rc)
    for t in outs.values():
        if t is not None:
            t.fill_(-7.0) if t.dtype == torch.float32 else t.fill_(-7)
    for _ in range(2):  # zeroed by the graph: two launches give one step's gradients
        assert L.sof_graph_launch(graph, side.cuda_stream) == L.SOF_OK
    side.synchronize()
    assert ws.stats()["n_dropped"] == 0
    L.sof_graph_destroy(graph)
    # reference: checked forward + backward per call of two views, on a fresh workspace
    ref_outs, ref_grads, ref_sg = buffers()
    ws2 = R.Workspace()
    checked = L.sof_render_opts.from_buffer_copy(best)
    checked.flags |= L.SOF_FLAG_CHECKED
    p0 = 0
    for i in range(0, len(cams), 2):
        sub = cams[i:i + 2]
        p1 = p0 + sum(c.width * c.height for c in sub)
        o = {k: (None if v is None else (v[3 * p0:3 * p1] if k in ("color", "normal") else v[p0:p1]))
             for k, v in ref_outs.items()}
        sub_c = R.cameras_to_c(sub)
        R.render_forward_raw(scene_c, sub_c, len(sub), checked, o, ws2)
        gi = L.sof_render_grad_in()
        gi.d_color, gi.d_opacity = d_color[3 * p0:3 * p1].data_ptr(), d_opacity[p0:p1].data_ptr()
        L.check(L.sof_render_bwd(scene_c, sub_c, len(sub), checked, R._out_c(o), gi, ref_sg, ws2.handle,
                                 torch.cuda.current_stream().cuda_stream), "sof_render_bwd", ws2.handle)
        p0 = p1
    torch.cuda.synchronize()
    for k, v in ref_outs.items():
        if v is not None:
            assert torch.equal(outs[k], v), k
    for x, y in zip(grads, ref_grads):
        assert float((x - y).abs().max()) <= 1e-5 * (float(y.abs().max()) + 1e-30)


def test_backward_needs_its_own_forward():
    from paper_2506_19139_gb300 import _lib as L
    from paper_2506_19139_gb300 import render as R
    scene = syn.uniform_box_scene(1500, 13, 1.0, (0.02, 0.2), (0.1, 0.99), 1)
    cams = _cams()
    ts = R.scene_tensors(scene, requires_grad=True)
    ws = R.Workspace()
    a = R.render(*ts, cams[:1], R.RenderOptions(), ws)
    b = R.render(*ts, cams[2:3], R.RenderOptions(), ws)
    with pytest.raises(RuntimeError):
        a["color"].sum().backward(retain_graph=True)
    b["color"].sum().backward()  # the last forward's backward is fine
    # the C-ABI refuses other cameras and other output buffers than its last forward's
    scene_c = R.scene_to_c(*[t.detach() for t in ts])
    opts = R.RenderOptions().to_c()
    gin = L.sof_render_grad_in()
    d = torch.ones(3 * cams[0].width * cams[0].height, device="cuda")
    gin.d_color = d.data_ptr()
    grads = [torch.zeros_like(t) for t in ts]
    sg = L.sof_scene_grad()
    sg.d_means, sg.d_log_scales, sg.d_quats = grads[0].data_ptr(), grads[1].data_ptr(), grads[2].data_ptr()
    sg.d_opacity_logits, sg.d_sh = grads[3].data_ptr(), grads[4].data_ptr()
    outs_a = R.alloc_outputs(cams[:1], "cuda")
    outs_b = R.alloc_outputs(cams[:1], "cuda")
    stream = torch.cuda.current_stream().cuda_stream
    R.render_forward_raw(scene_c, R.cameras_to_c(cams[:1]), 1, opts, outs_a, ws)
    R.render_forward_raw(scene_c, R.cameras_to_c(cams[:1]), 1, opts, outs_b, ws)
    assert L.sof_render_bwd(scene_c, R.cameras_to_c(cams[:1]), 1, opts, R._out_c(outs_a), gin, sg, ws.handle,
                            stream) == L.SOF_ERR_STATE
    assert L.sof_render_bwd(scene_c, R.cameras_to_c(cams[1:2]), 1, opts, R._out_c(outs_b), gin, sg, ws.handle,
                            stream) == L.SOF_ERR_STATE
    assert L.sof_render_bwd(scene_c, R.cameras_to_c(cams[:1]), 1, opts, R._out_c(outs_b), gin, sg, ws.handle,
                            stream) == L.SOF_OK
    torch.cuda.synchronize()


def test_reservation_sizes_the_stream_ordered_forward_exactly():
    """sof_workspace_reserve counts the pairs that pass the tile test (far fewer than the tested
    items a checked forward reserves a pair for): the reserved workspace is smaller than the checked
    forward's, the stream-ordered forward on it drops nothing, and its images equal the checked
    forward's."""
    from paper_2506_19139_gb300 import _lib as L
    from paper_2506_19139_gb300 import render as R
    scene = syn.uniform_box_scene(3000, 14, 1.0, (0.02, 0.3), (0.1, 0.99), 1)
    cams = _cams()
    ts = R.scene_tensors(scene)
    scene_c, cams_c = R.scene_to_c(*ts), R.cameras_to_c(cams)
    checked = R.Workspace()
    ref = R.alloc_outputs(cams, "cuda")
    R.render_forward_raw(scene_c, cams_c, len(cams), R.RenderOptions().to_c(), ref, checked)
    ws = R.Workspace()
    opts = R.RenderOptions(async_mode=True).to_c()
    reserved = ws.reserve(scene_c, cams_c, len(cams), opts)
    assert reserved < checked.buffer.numel()
    got = R.alloc_outputs(cams, "cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):
        assert L.sof_render_fwd(scene_c, cams_c, len(cams), opts, R._out_c(got), ws.handle, stream) == L.SOF_OK
    torch.cuda.synchronize()
    st = ws.stats()
    assert st["n_dropped"] == 0
    for k, v in ref.items():
        if v is not None:
            assert torch.equal(got[k], v), k
