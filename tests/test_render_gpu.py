"""GPU parity of the forward render against the FP64 oracle, element by element over whole images:
every pixel inside the oracle's interval of correct results (tests/parity.py states the tolerances
and what may be left out, which is counted and bounded).
"""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2506_19139_gb300 import synthetic as syn
from parity import check_bounds, flat

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2506_19139_gb300 import build
    build.build()


def _gpu_render(scene, cams, **kw):
    from paper_2506_19139_gb300 import render as R
    ts = R.scene_tensors(scene)
    opts = R.RenderOptions(**kw)
    res = R.render(*ts, cams, opts)
    torch.cuda.synchronize()
    imgs = R.view_images(res, cams)
    stats = res["workspace"].stats()
    return [{k: v.detach().cpu().numpy() for k, v in im.items()} for im in imgs], stats


def compare(gpu, ref, label, **kw):
    """Whole images: gpu from view_images(), ref from oracle.render(..., bounds=True)."""
    r = {"flags": ref["flags"], "exact_sens": ref["exact_sens"]}
    for side in ("lo", "hi"):
        r[side] = {k: (v.reshape(3, -1).T if k in ("color", "normal") else v.reshape(-1)) for k, v in ref[side].items()}
    return check_bounds(flat(gpu), r, label, **kw)


def test_tiny_forward_matches_oracle():
    """1,000 Gaussians, one 64x64 camera at distance 4 (the tiny configuration)."""
    scene, cams = syn.tiny_forward(0)
    gpu, stats = _gpu_render(scene, cams)
    ref = oracle.render(scene, cams[0], bounds=True)
    compare(gpu[0], ref, "tiny")
    assert stats["inexact_pixels"] == 0
    assert (ref["n_contrib"] > 0).mean() > 0.25


@pytest.mark.parametrize("seed,tile", [(1, 16), (2, 16), (1, 8), (2, 32)])
def test_ragged_tiles_and_background(seed, tile):
    """Image sizes that are not multiples of the tile, a non-zero background, several seeds, tiles
    of 8, 16 and 32 pixels."""
    scene = syn.uniform_box_scene(1500, seed, 1.0, (0.01, 0.2), (0.1, 0.99), 1)
    cam = syn.look_at((0.5, -0.3, 3.5), (0.0, 0.1, 0.0), 75, 45, 55.0)
    gpu, stats = _gpu_render(scene, [cam], bg=(0.2, 0.1, 0.7), tile=tile)
    ref = oracle.render(scene, cam, bg=(0.2, 0.1, 0.7), bounds=True)
    compare(gpu[0], ref, f"ragged{seed} tile {tile}")
    assert stats["inexact_pixels"] == 0


def test_multi_view_packed_outputs():
    """Three views of different sizes in one call; each equals its own oracle render."""
    scene = syn.uniform_box_scene(800, 5, 1.0, (0.02, 0.15), (0.1, 0.99), 2)
    cams = [syn.look_at((3.5 * math.sin(a), 0.4, 3.5 * math.cos(a)), (0, 0, 0), w, h, 60.0)
            for a, (w, h) in zip((0.0, 2.1, 4.2), ((48, 40), (33, 64), (80, 17)))]
    gpu, stats = _gpu_render(scene, cams)
    for i, cam in enumerate(cams):
        compare(gpu[i], oracle.render(scene, cam, bounds=True), f"view{i}")


@pytest.mark.parametrize("tile,k", [(16, 16), (8, 16), (32, 8), (16, 8)])
def test_dense_overlap_needs_exact_order(tile, k):
    """Large overlapping Gaussians near the camera: many hits per pixel with close t*, so the
    per-pixel reorder is exercised (a tile-level sort alone would be wrong here). With small
    buffers many pixels overflow: the second pass (tiles of 8 and 16) or directly the fallback
    (tiles of 32) recompute them."""
    scene = syn.uniform_box_scene(400, 9, 0.8, (0.05, 0.5), (0.05, 0.6), 0)
    cam = syn.look_at((0.0, 0.0, 2.2), (0.0, 0.0, 0.0), 64, 48, 70.0)
    gpu, stats = _gpu_render(scene, [cam], tile=tile, reorder_k=k)
    ref = oracle.render(scene, cam, bounds=True)
    compare(gpu[0], ref, f"dense tile {tile} k {k}")
    if k == 8:
        assert stats["n_forced"] > 0
    assert ref["n_contrib"].mean() > 8
    assert stats["inexact_pixels"] == 0


def test_median_depth_and_near_plane():
    """Median (GOF) depth channel, and a camera inside the cloud so that the near plane cuts."""
    scene = syn.uniform_box_scene(1200, 12, 1.0, (0.02, 0.2), (0.1, 0.99), 0)
    cam = syn.look_at((0.1, 0.05, 0.3), (0.0, 0.0, -3.0), 40, 40, 80.0)
    gpu, stats = _gpu_render(scene, [cam], median_depth=True)
    ref = oracle.render(scene, cam, bounds=True)
    compare(gpu[0], ref, "inside", median=True)


def test_empty_dead_and_nonfinite_gaussians():
    """No Gaussians -> background; dead (o <= 1/255) and NaN Gaussians are culled."""
    scene, cams = syn.tiny_forward(0, n=50)
    empty = scene.subset(np.arange(0))
    gpu, _ = _gpu_render(empty, cams, bg=(0.3, 0.4, 0.5))
    assert np.allclose(gpu[0]["color"], np.array([0.3, 0.4, 0.5])[:, None, None])
    assert np.all(gpu[0]["opacity"] == 0) and np.all(gpu[0]["n_contrib"] == 0)
    bad = scene.subset(np.arange(50))
    bad.opacity_logits[:10] = -20.0          # dead
    bad.means[10:12] = np.nan                # non-finite
    gpu, stats = _gpu_render(bad, cams)
    clean = bad.subset(np.arange(12, 50))
    clean_gpu, _ = _gpu_render(clean, cams)
    np.testing.assert_array_equal(gpu[0]["n_contrib"], clean_gpu[0]["n_contrib"])
    np.testing.assert_allclose(gpu[0]["color"], clean_gpu[0]["color"], atol=1e-6)
    assert stats["nonfinite"] == 2


def test_view_without_gaussians_in_a_multi_view_call():
    """One call of three views, the middle one looking away from every Gaussian: that view is the
    background with no hits, the others equal their single-view renders bit for bit, and a loss over
    all three gives the gradients of the two non-empty views alone."""
    from paper_2506_19139_gb300 import render as R
    scene = syn.uniform_box_scene(600, 9, 1.0, (0.02, 0.15), (0.1, 0.99), 1)
    cams = [syn.look_at((0.0, 0.3, 3.5), (0.0, 0.0, 0.0), 40, 32, 60.0),
            syn.look_at((0.0, 0.0, 6.0), (0.0, 0.0, 12.0), 24, 24, 60.0),   # looking away
            syn.look_at((3.5, 0.2, 0.0), (0.0, 0.0, 0.0), 32, 40, 60.0)]
    bg = (0.25, 0.5, 0.75)
    gpu, stats = _gpu_render(scene, cams, bg=bg)
    assert np.allclose(gpu[1]["color"], np.array(bg)[:, None, None])
    assert np.all(gpu[1]["opacity"] == 0) and np.all(gpu[1]["n_contrib"] == 0)
    for i in (0, 2):
        single, _ = _gpu_render(scene, [cams[i]], bg=bg)
        for k in ("color", "depth", "opacity", "n_contrib", "exact_depth"):
            np.testing.assert_array_equal(gpu[i][k], single[0][k])

    def grads(cam_list):
        ts = R.scene_tensors(scene, requires_grad=True)
        res = R.render(*ts, cam_list, R.RenderOptions(bg=bg))
        imgs = R.view_images(res, cam_list)
        loss = sum((im["color"] * (j + 1)).sum() + im["opacity"].sum() for j, im in enumerate(imgs))
        loss.backward()
        return [t.grad.detach().cpu().numpy() for t in ts]

    g_all = grads(cams)
    g0 = grads([cams[0]])
    ts2 = R.scene_tensors(scene, requires_grad=True)
    res2 = R.render(*ts2, [cams[2]], R.RenderOptions(bg=bg))
    im2 = R.view_images(res2, [cams[2]])[0]
    ((im2["color"] * 3).sum() + im2["opacity"].sum()).backward()
    g2 = [t.grad.detach().cpu().numpy() for t in ts2]
    for a, b, c in zip(g_all, g0, g2):
        np.testing.assert_allclose(a, b + c, rtol=1e-4, atol=1e-6 * max(1.0, float(np.abs(b + c).max())))


def test_degenerate_image_sizes():
    """Views of 1x1, 1x37 and 37x1 pixels in one call (tiles mostly outside the image); each
    equals its own oracle render."""
    scene = syn.uniform_box_scene(400, 13, 1.0, (0.05, 0.3), (0.2, 0.99), 0)
    cams = [syn.look_at((0.2, 0.1, 3.0), (0.0, 0.0, 0.0), w, h, 30.0) for w, h in ((1, 1), (1, 37), (37, 1))]
    gpu, stats = _gpu_render(scene, cams, bg=(0.1, 0.2, 0.3))
    for i, cam in enumerate(cams):
        compare(gpu[i], oracle.render(scene, cam, bg=(0.1, 0.2, 0.3), bounds=True), f"degenerate view {i}")
    assert stats["inexact_pixels"] == 0
    assert sum(int((g["n_contrib"] > 0).sum()) for g in gpu) > 10


def test_needles_and_pancakes():
    """Strongly anisotropic Gaussians (axis ratios of 100: needles of 0.01 x 0.01 x 1 and pancakes of
    0.005 x 0.5 x 0.5) in random orientations; every pixel within the oracle's interval. (At ratios
    of 500 the FP32 weights drift to about 1e-5 of the normal and colour, the tolerance itself.)"""
    rng = np.random.default_rng(17)
    n = 300
    scales = np.where(rng.random((n, 1)) < 0.5, np.array([[0.01, 0.01, 1.0]]), np.array([[0.005, 0.5, 0.5]]))
    scene = syn.uniform_box_scene(n, 17, 1.0, (0.05, 0.1), (0.2, 0.99), 0)
    scene.log_scales[:] = np.log(scales * rng.uniform(0.5, 1.5, (n, 1))).astype(np.float32)
    cam = syn.look_at((0.4, 0.9, 3.2), (0.0, 0.0, 0.0), 96, 72, 60.0)
    gpu, stats = _gpu_render(scene, [cam])
    ref = oracle.render(scene, cam, bounds=True)
    compare(gpu[0], ref, "needles and pancakes")
    assert stats["inexact_pixels"] == 0
    assert (ref["n_contrib"] > 0).mean() > 0.2


@pytest.mark.parametrize("t_stop,near", [(0.0, 0.2), (0.3, 0.2), (1e-4, 1.5)])
def test_stop_threshold_and_near_plane_extremes(t_stop, near):
    """No early stop at all (every hit composited, up to about 200 per pixel), an early stop at
    T = 0.3, and a near plane inside the scene; every pixel within the oracle's interval. The
    backward (with 64-entry replay lists, so that long pixels are re-merged) gives finite gradients
    and replays no more hits than the forward composited."""
    from paper_2506_19139_gb300 import render as R
    scene = syn.uniform_box_scene(2500, 19, 1.0, (0.03, 0.2), (0.2, 0.99), 0)
    cam = syn.look_at((0.3, 0.2, 3.0), (0.0, 0.0, 0.0), 48, 40, 60.0)
    gpu, stats = _gpu_render(scene, [cam], t_stop=t_stop, near_plane=near)
    ref = oracle.render(scene, cam, near=near, t_stop=t_stop, bounds=True)
    compare(gpu[0], ref, f"t_stop {t_stop} near {near}")
    assert stats["inexact_pixels"] == 0 and stats["n_below_key"] == 0
    ts = R.scene_tensors(scene, requires_grad=True)
    res = R.render(*ts, [cam], R.RenderOptions(t_stop=t_stop, near_plane=near, replay_cap=64))
    R.view_images(res, [cam])[0]["color"].sum().backward()
    assert all(torch.isfinite(t.grad).all() for t in ts)
    st = res["workspace"].stats()
    assert st["n_replayed"] <= st["n_composited"]


def test_second_pass_in_two_sweeps():
    """Faint, wide Gaussians in front of the camera: with 8-entry buffers more than half of the
    pixels overflow the first pass, so some 16x16 tile hands more than 128 pixels to the second
    pass, which holds 64-entry buffers for 128 pixels at a time and takes them in two sweeps. The
    redone pixels (and the fallback's) stay within the oracle's interval, and the backward's own
    merge gives the recorded order's gradients."""
    from paper_2506_19139_gb300 import render as R
    scene = syn.uniform_box_scene(3000, 24, 0.8, (0.1, 0.4), (0.05, 0.3), 0)
    cam = syn.look_at((0.0, 0.0, 2.4), (0.0, 0.0, 0.0), 48, 32, 70.0)
    gpu, stats = _gpu_render(scene, [cam], tile=16, reorder_k=8)
    assert stats["n_forced"] > 128 * 6  # 6 tiles: one of them holds more than 128
    compare(gpu[0], oracle.render(scene, cam, bounds=True), "two sweeps")
    assert stats["inexact_pixels"] == 0
    grads = []
    for cap in (256, -1):
        ts = R.scene_tensors(scene, requires_grad=True)
        res = R.render(*ts, [cam], R.RenderOptions(tile=16, reorder_k=8, replay_cap=cap))
        img = R.view_images(res, [cam])[0]
        (img["color"].sum() + img["depth"].sum()).backward()
        grads.append([t.grad.detach().double().cpu().numpy() for t in ts])
    for a, b in zip(*grads):
        assert np.linalg.norm(a - b) <= 1e-5 * max(np.linalg.norm(a), 1e-30)
