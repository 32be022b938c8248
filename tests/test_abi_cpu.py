"""CPU-side checks of the C-ABI library: it builds for sm_103a, loads, and exports every entry
point declared in include/sof.h (no compute call needs a GPU here)."""
import ctypes
import os
import re

import pytest

from paper_2506_19139_gb300 import _lib, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "sof.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sof_[a-z0-9_]+)\s*\(", src)))


def test_library_builds_and_exports_every_declared_symbol():
    path = build.build()
    assert os.path.exists(path)
    lib = ctypes.CDLL(path)
    names = _declared()
    assert "sof_render_fwd" in names and "sof_render_bwd" in names and "sof_opacity_query" in names
    for n in names:
        assert hasattr(lib, n), n
    # the Python binding covers the same names
    assert set(names) <= set(_lib.SIGNATURES)


def test_error_paths_without_gpu():
    lib = _lib.load()
    assert lib.sof_version() >= 1
    assert lib.sof_error_string(_lib.SOF_ERR_WORKSPACE_TOO_SMALL) == b"workspace too small"
    h = _lib.sof_workspace_create()
    try:
        # invalid arguments are rejected before any device work
        scene = _lib.sof_scene()
        scene.n = -1
        cams = (_lib.sof_camera * 1)()
        opts = _lib.sof_render_opts()
        out = _lib.sof_render_out()
        assert _lib.sof_render_fwd(scene, cams, 1, opts, out, h, 0) == _lib.SOF_ERR_INVALID_ARG
        scene.n = 0
        assert _lib.sof_render_fwd(scene, cams, 0, opts, out, h, 0) == _lib.SOF_ERR_INVALID_ARG
        assert lib.sof_workspace_bind(h, ctypes.c_void_p(17), 100) == _lib.SOF_ERR_INVALID_ARG
        gin = _lib.sof_render_grad_in()
        sg = _lib.sof_scene_grad()
        assert _lib.sof_render_bwd(scene, cams, 1, opts, out, gin, sg, h, 0) in (_lib.SOF_ERR_STATE,
                                                                                  _lib.SOF_ERR_INVALID_ARG)
    finally:
        _lib.sof_workspace_destroy(h)


def test_workspace_size_grows_with_pairs():
    scene = _lib.sof_scene()
    scene.n = 1000
    scene.sh_degree = 0
    scene.means = scene.log_scales = scene.quats = scene.opacity_logits = scene.sh = 256
    cams = (_lib.sof_camera * 1)()
    cams[0].width = cams[0].height = 64
    cams[0].fx = cams[0].fy = 55.0
    cams[0].cx = cams[0].cy = 32.0
    for i in (0, 5, 10):
        cams[0].world_to_cam[i] = 1.0
    opts = _lib.sof_render_opts()
    opts.near_plane, opts.t_stop = 0.2, 1e-4
    a = _lib.sof_render_workspace_size(scene, cams, 1, opts, 1000)
    b = _lib.sof_render_workspace_size(scene, cams, 1, opts, 100000)
    assert b - a >= 99000 * 20 - 4 * 256  # per pair: 12 B unsorted (tile, key, record) + 8 B tile-sorted word


def _valid_inputs():
    scene = _lib.sof_scene()
    scene.n = 1000
    scene.sh_degree = 0
    scene.means = scene.log_scales = scene.quats = scene.opacity_logits = scene.sh = 256
    cams = (_lib.sof_camera * 2)()
    for c in cams:
        c.width, c.height = 64, 48
        c.fx = c.fy = 55.0
        c.cx, c.cy = 32.0, 24.0
        for i in (0, 5, 10):
            c.world_to_cam[i] = 1.0
        c.world_to_cam[11] = 4.0
    opts = _lib.sof_render_opts()
    opts.near_plane, opts.t_stop = 0.2, 1e-4
    opts.tile, opts.chunk, opts.reorder_k, opts.replay_cap = 16, 64, 16, 256
    return scene, cams, opts


@pytest.mark.parametrize("field,value", [
    ("scene.n", -1), ("scene.sh_degree", 4), ("scene.quats", 260),            # unaligned quaternions
    ("cam.width", 0), ("cam.height", 70000), ("cam.fx", 0.0), ("cam.world_to_cam3", float("nan")),
    ("opts.tile", 12), ("opts.chunk", 48), ("opts.reorder_k", 4), ("opts.t_stop", 1.0),
    ("opts.near_plane", -0.1), ("opts.replay_cap", 5000), ("opts.sort_prefix", -2),
    ("n_views", 0)])
def test_invalid_render_arguments_are_refused_before_device_work(field, value):
    """Every argument the header states a range for is checked before any device work: the
    workspace-size query (no GPU needed) refuses it with SOF_ERR_INVALID_ARG."""
    scene, cams, opts = _valid_inputs()
    n_views = 2
    assert _lib.sof_render_workspace_size(scene, cams, n_views, opts, 1000) > 0  # the valid call
    obj, name = field.split(".") if "." in field else ("", field)
    if obj == "scene":
        setattr(scene, name, value)
    elif obj == "opts":
        setattr(opts, name, value)
    elif obj == "cam":
        if name.startswith("world_to_cam"):
            cams[1].world_to_cam[int(name[len("world_to_cam"):])] = value
        else:
            setattr(cams[1], name, value)
    else:
        n_views = value
    with pytest.raises(_lib.SOFError) as e:
        _lib.sof_render_workspace_size(scene, cams, n_views, opts, 1000)
    assert e.value.code == _lib.SOF_ERR_INVALID_ARG


@pytest.mark.parametrize("field,value", [("tile", 12), ("flags", 1 << 7), ("t_stop_query", 1.0),
                                         ("near_plane", -1.0), ("n_points", -1)])
def test_invalid_query_arguments_are_refused_before_device_work(field, value):
    scene, cams, _ = _valid_inputs()
    q = _lib.sof_query_opts()
    q.near_plane, q.t_stop_query, q.tile, q.flags = 0.2, 0.0, 16, 0
    n_points = 100
    assert _lib.sof_query_workspace_size(scene, cams, 2, n_points, q, 1000) > 0
    if field == "n_points":
        n_points = value
    else:
        setattr(q, field, value)
    with pytest.raises(_lib.SOFError) as e:
        _lib.sof_query_workspace_size(scene, cams, 2, n_points, q, 1000)
    assert e.value.code == _lib.SOF_ERR_INVALID_ARG
