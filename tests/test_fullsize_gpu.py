"""Parity at the full workload sizes, in the launch configuration the benchmark times, on sampled
outputs the FP64 oracle computes one by one:

- the 1M-Gaussian unbounded scene at 1920x1080 (forward outputs at 1024 random pixels, plus the
  backward's bookkeeping: the pixels within the replay capacity are replayed hit for hit);
- the differentiable-step scene (100K Gaussians, SH degree 3, four 256x256 views in one call) at 256
  random pixels per view;
- the meshing query (3M Gaussians, 27M points, 100 views at 1000x750) at random points, each
  within the oracle's interval of correct results;
- a camera inside and among Gaussians, where the per-Gaussian and per-tile near-plane bounds cull
  records that could never pass the t* > near test (full image).

Tolerances as in test_render_gpu / test_query_gpu: 1e-5 absolute on colour, opacity and normal,
1e-4 relative on depth, plus the oracle's slack where two hits are near-tied in t*; pixels flagged
by other margins are excluded and counted.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2506_19139_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2506_19139_gb300 import build
    build.build()


def _check_pixels(gpu, ref, pix, W, H, label, max_flag_frac=5e-2):
    """gpu: per-view images from view_images(); ref: oracle.render(..., pixels=pix). Near ties in
    t* are checked with the oracle's slack for the swap. A 0.5 crossing within the margin only
    affects the exact depth. Pixels with other margin flags (an alpha at 1/255, a t* at the near
    plane, a transmittance at the stop) are excluded from the strict check, counted, and checked
    only for plausibility: at full size each pixel weighs hundreds of candidates, so a few percent
    of pixels meet one such decision."""
    depth_only = oracle.FLAG_EXACT | oracle.FLAG_CROSS
    F = ref["flags"] & ~depth_only
    ok = (F & ~oracle.FLAG_ORDER) == 0
    assert (~ok).sum() <= max(2, max_flag_frac * len(pix)), f"{label}: {int((~ok).sum())} flagged"
    op_all = gpu["opacity"].reshape(-1)[pix]
    assert (np.abs(op_all - ref["opacity"])[~ok] <= 0.05).all(), label
    assert (np.abs(gpu["n_contrib"].reshape(-1)[pix] - ref["n_contrib"])[~ok] <= 3).all(), label
    col = gpu["color"].reshape(3, -1)[:, pix].T
    nrm = gpu["normal"].reshape(3, -1)[:, pix].T
    op = gpu["opacity"].reshape(-1)[pix]
    dep = gpu["depth"].reshape(-1)[pix]
    cnt = gpu["n_contrib"].reshape(-1)[pix]
    assert (np.abs(col - ref["color"]).max(1) <= 1e-5 + ref["slack_color"])[ok].all(), label
    assert (np.abs(nrm - ref["normal"]).max(1) <= 1e-5 + ref["slack_normal"])[ok].all(), label
    assert np.abs(op - ref["opacity"])[ok].max() <= 1e-5, label
    D, O = ref["depth"], ref["opacity"]
    tol_d = 1e-4 * np.abs(D) + 1e-5 * D / np.maximum(O, 1e-6) + 1e-7 + ref["slack_depth"]
    assert (np.abs(dep - D) <= tol_d)[ok].all(), label
    np.testing.assert_array_equal(cnt[ok], ref["n_contrib"][ok], err_msg=label)
    ex_ok = ok & ((ref["flags"] & depth_only) == 0)
    ex = gpu["exact_depth"].reshape(-1)[pix]
    assert (np.abs(ex - ref["exact_depth"]) <= 1e-4 * np.abs(ref["exact_depth"]) + 1e-7)[ex_ok].all(), label


def test_unbounded_1m_1080p_sampled_pixels_and_replay_bookkeeping():
    from paper_2506_19139_gb300 import render as R
    scene, cams = syn.unbounded_training()
    cam = cams[0]
    ts = R.scene_tensors(scene, requires_grad=True)
    res = R.render(*ts, cams, R.RenderOptions())
    img = R.view_images(res, cams)[0]
    loss = img["color"].sum() + 0.1 * img["depth"].sum() + img["opacity"].sum()
    loss.backward()
    torch.cuda.synchronize()
    st = res["workspace"].stats()
    assert st["inexact_pixels"] == 0 and st["n_below_key"] == 0 and st["n_unsorted"] == 0
    for t in ts:
        assert torch.isfinite(t.grad).all()
    gpu = {k: v.detach().cpu().numpy() for k, v in img.items() if v is not None}
    # pixels with at most replay_cap hits are replayed, the others re-merged by the backward
    cnt = gpu["n_contrib"].astype(np.int64)
    assert st["n_composited"] == int(cnt.sum())
    assert st["n_replayed"] == int(cnt[cnt <= R.RenderOptions().replay_cap].sum())
    rng = np.random.default_rng(7)
    pix = rng.choice(cam.width * cam.height, 1024, replace=False).astype(np.int64)
    ref = oracle.render(scene, cam, pixels=pix)
    assert (ref["n_contrib"] > 0).mean() > 0.9
    _check_pixels(gpu, ref, pix, cam.width, cam.height, "unbounded-1080p")


def test_differentiable_step_100k_four_views_sampled_pixels():
    from paper_2506_19139_gb300 import render as R
    scene, cams = syn.differentiable_step()
    ts = R.scene_tensors(scene)
    with torch.no_grad():
        res = R.render(*ts, cams, R.RenderOptions())
    imgs = R.view_images(res, cams)
    rng = np.random.default_rng(8)
    for v, cam in enumerate(cams):
        gpu = {k: t.cpu().numpy() for k, t in imgs[v].items() if t is not None}
        pix = rng.choice(cam.width * cam.height, 256, replace=False).astype(np.int64)
        ref = oracle.render(scene, cam, pixels=pix)
        _check_pixels(gpu, ref, pix, cam.width, cam.height, f"diffstep-view{v}")


def test_meshing_query_3m_27m_points_100_views_sampled_points():
    from paper_2506_19139_gb300 import render as R
    scene, cams, pts = syn.meshing_query()
    ts = R.scene_tensors(scene)
    ws = R.Workspace()
    o, s = R.opacity_query(ts[0], ts[1], ts[2], ts[3], cams, torch.as_tensor(pts, device="cuda"),
                           R.QueryOptions(), ws)
    torch.cuda.synchronize()
    o, s = o.cpu().numpy(), s.cpu().numpy()
    st = ws.stats()
    assert st["n_point_views"] == int(s.astype(np.int64).sum())
    idx = np.random.default_rng(9).choice(len(pts), 6, replace=False)
    ref = oracle.query(scene, cams, pts[idx])
    # every sampled point lies within the oracle's interval of correct results (P11)
    assert (o[idx] >= ref["lo"] - 1e-5).all() and (o[idx] <= ref["hi"] + 1e-5).all()
    assert (np.abs(s[idx] - ref["seen"]) <= ref["maybe_seen"]).all()
    tight = ref["hi"] - ref["lo"] <= 1e-12
    assert np.abs(o[idx] - ref["opacity"])[tight].max(initial=0.0) <= 1e-5


def test_camera_inside_and_among_gaussians_near_plane_culling():
    """Large Gaussians around the camera: some contain it (their t* never exceeds the near
    plane in some directions), some straddle the image plane. The culled GPU path must equal the
    oracle, which evaluates every Gaussian at every pixel."""
    rng = np.random.default_rng(11)
    n = 400
    means = rng.normal(0.0, 0.35, (n, 3))
    means[:40] = rng.normal(0.0, 0.05, (40, 3))            # right around the camera
    log_s = np.log(rng.uniform(0.03, 0.4, (n, 3)))
    q = rng.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    opac = rng.uniform(0.2, 0.95, n)
    sh = np.zeros((n, 1, 3))
    sh[:, 0, :] = (rng.uniform(0, 1, (n, 3)) - 0.5) / 0.28209479177387814
    f32 = lambda a: np.ascontiguousarray(a, dtype=np.float32)
    scene = syn.Scene(f32(means), f32(log_s), f32(q), f32(np.log(opac / (1 - opac))), f32(sh), 0)
    cam = syn.look_at((0.0, 0.0, 0.0), (0.3, 0.1, 1.0), 72, 56, 90.0)
    from paper_2506_19139_gb300 import render as R
    ts = R.scene_tensors(scene)
    with torch.no_grad():
        res = R.render(*ts, [cam], R.RenderOptions())
    gpu = {k: t.cpu().numpy() for k, t in R.view_images(res, [cam])[0].items() if t is not None}
    pix = np.arange(cam.width * cam.height, dtype=np.int64)
    ref = oracle.render(scene, cam, pixels=pix, cull=False)
    assert (ref["n_contrib"] > 0).mean() > 0.5
    _check_pixels(gpu, ref, pix, cam.width, cam.height, "inside", max_flag_frac=1e-2)
