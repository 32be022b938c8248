"""The sorted front of the tiles' lists (sort_prefix): the composite's first pass reads only the
smallest keys of each tile, and pixels still open where the front ends are redone after the rest of
the list is sorted. The result must not depend on the front's size:

- images bit-identical to whole-list sorting (n_open counts the pixels redone), for fronts from a few entries (most pixels redone)
  to the default, with the recorded order (replay) and with the backward's own merge;
- gradients equal up to the order of float atomics;
- a tile of 8000 entries with 6000 equal keys: the front cannot be cut inside the equal keys, so it
  is longer than one shared-memory block and goes through the long-list sort.
"""
import numpy as np
import pytest
import torch

from paper_2506_19139_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2506_19139_gb300 import build
    build.build()


def _run(scene, cams, prefix, replay_cap=256, reorder_k=16, seed=0):
    from paper_2506_19139_gb300 import render as R
    ts = R.scene_tensors(scene, requires_grad=True)
    res = R.render(*ts, cams, R.RenderOptions(sort_prefix=prefix, replay_cap=replay_cap, reorder_k=reorder_k))
    st = res["workspace"].stats()
    imgs = R.view_images(res, cams)
    g = torch.Generator(device="cuda").manual_seed(seed)
    loss = 0.0
    for im in imgs:
        for k in ("color", "depth", "normal", "opacity"):
            loss = loss + (torch.randn(im[k].shape, device="cuda", generator=g) * im[k]).sum()
    loss.backward()
    outs = [{k: v.detach().cpu().numpy() for k, v in im.items()} for im in imgs]
    return outs, [t.grad.detach().double().cpu().numpy() for t in ts], st


def _same(ref, got, label):
    outs_a, grads_a, _ = ref
    outs_b, grads_b, st = got
    for v, (a, b) in enumerate(zip(outs_a, outs_b)):
        for k in a:
            np.testing.assert_array_equal(b[k], a[k], err_msg=f"{label} view {v} {k}")
    for a, b in zip(grads_a, grads_b):
        assert np.linalg.norm(a - b) <= 1e-5 * max(np.linalg.norm(a), 1e-30), label
    assert st["inexact_pixels"] == 0 and st["n_unsorted"] == 0 and st["n_below_key"] == 0, label


@pytest.mark.parametrize("replay_cap,reorder_k", [(256, 16), (-1, 16), (256, 8)])
def test_front_size_changes_nothing(replay_cap, reorder_k):
    """With reorder_k = 8 many pixels overflow the first pass's buffer; the second pass then reads
    the front only in tiles without open pixels, and its own open pixels go to the fallback."""
    scene = syn.uniform_box_scene(4000, 5, 1.0, (0.02, 0.25), (0.2, 0.99), 3)
    cams = [syn.look_at((0.3, -0.2, 3.0), (0.0, 0.0, 0.0), 96, 80, 55.0),
            syn.look_at((-2.0, 0.5, 2.2), (0.0, 0.0, 0.0), 70, 45, 60.0)]
    ref = _run(scene, cams, -1, replay_cap, reorder_k)
    assert ref[2]["n_open"] == 0
    opened = {}
    for prefix in (1, 8, 100, 300, 0):
        got = _run(scene, cams, prefix, replay_cap, reorder_k)
        _same(ref, got, f"prefix {prefix}")
        opened[prefix] = got[2]["n_open"]
        assert got[2]["n_read"] <= ref[2]["n_read"]
    assert opened[1] > 0 and opened[8] > 0


def test_front_of_equal_keys_longer_than_one_block():
    n_eq, n_far = 6000, 2000
    base = syn.uniform_box_scene(n_eq + n_far, 6, 1.0, (0.3, 0.3), (0.02, 0.02), 0)
    means = np.zeros((n_eq + n_far, 3), np.float32)
    means[n_eq:, 2] = -2.0  # behind the equal-key stack, seen from +z
    quats = np.tile(np.array([1.0, 0.0, 0.0, 0.0], np.float32), (n_eq + n_far, 1))
    scene = syn.Scene(means, base.log_scales, quats, base.opacity_logits, base.sh, 0)
    cams = [syn.look_at((0.0, 0.0, 3.0), (0.0, 0.0, 0.0), 32, 32, 40.0)]
    ref = _run(scene, cams, -1)
    for prefix in (64, 0):
        _same(ref, _run(scene, cams, prefix), f"prefix {prefix}")
